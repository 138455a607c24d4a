// Batched shifted COCG driver: many (problem, shift) slots advanced together.
#pragma once

#include <cuda.h>

#include "tem_internal.h"

namespace tem {

// Vectors of one slot (pointers into a batch-owned allocation).
struct SlotVectors {
  void* x64[2];                                   // FP64 iterate (double-buffered)
  void* x; void* w; void* a0; void* a1; void* q;  // inner edge vectors
  void* xn; void* psi; void* b0; void* b1; void* cn; void* u; void* gp;  // inner nodal vectors
};

// Per-slot bytes of the vectors for one grid with `ncomp` entries per direction.
size_t slot_vector_bytes(int64_t ncomp, int precision);
// Carve the vectors of one slot out of `base` (slot_vector_bytes long, 256-aligned).
SlotVectors carve_slot(void* base, int64_t ncomp, int precision);

struct SolveStats {
  int launches = 0;     // kernels launched by the solve
  int outer_steps = 0;
};

// Sizes of the block lists: stencil (s blocks, the first s_fast of slots with tma), update (u,
// u_fast likewise), nodal (n).
struct BlockCounts {
  int s = 0, s_fast = 0, u = 0, u_fast = 0, n = 0;
};

class Batch {
 public:
  // Slots must be added before setup(); all share one precision.
  Batch(int precision, int nodal) : precision_(precision), nodal_(nodal) {}
  ~Batch();
  int add_slot(const GridView& g, double xi_re, double xi_im, const SlotVectors& v,
               const double* f_real, const void* rhs_complex, int rhs_div = 0);
  int setup(const tem_options& opt, cudaStream_t st, const double* ff_per_slot);
  int solve(const tem_options& opt, cudaStream_t st, SolveStats* stats);
  // host copies after solve()
  int fetch_scalars(cudaStream_t st);
  const std::vector<SlotScalars>& scalars() const { return sc_h_; }
  const SlotDesc* slots_device() const { return slots_d_.as<SlotDesc>(); }
  const SlotScalars* scalars_device() const { return sc_d_.as<SlotScalars>(); }
  int nslots() const { return (int)slots_h_.size(); }
  const std::vector<SlotDesc>& slots_host() const { return slots_h_; }
  int precision() const { return precision_; }

  int stencil_blocks() const { return bc_.s; }
  int update_blocks() const { return bc_.u; }
  int nodal_blocks() const { return bc_.n; }
  // launch one (stencil, update) pair or one residual pass for all slots (bench / profiling)
  int launch_iteration(cudaStream_t st);
  int launches_per_iteration() const;
  int launch_stencil(cudaStream_t st);
  int launch_update(cudaStream_t st);
  int launch_nodal(cudaStream_t st, int init_only);
  int launch_residual(cudaStream_t st);
  bool uses_tma() const { return bc_.s_fast > 0; }

 private:
  int drop_done_slots(cudaStream_t st);
  int precision_;
  int nodal_;
  std::vector<SlotDesc> slots_h_;
  std::vector<SlotScalars> sc_h_;
  BlockCounts bc_;
  int part_stride_ = 0;
  DevBuf slots_d_, sc_d_, map_d_, part_d_, ticket_d_, counters_d_, tmaps_d_;
  std::vector<char> used_;      // slots in the block lists
  int* counters_h_ = nullptr;   // pinned: [n_active, n_done]
};

struct BatchArgs;

// Interleaved block lists (stencil | update | nodal) of the slots with use[q] != 0.
void build_block_maps(const std::vector<SlotDesc>& slots, const std::vector<char>& use, std::vector<int2>& map,
                      BlockCounts* bc);
// FP32 passes A and B over the block lists: the TMA stencil and the 16-byte update over the
// slots with tma, the cp.async stencil and the scalar update over the others (one launch each
// part that has blocks).  Returns a status; counts its launches.
int launch_pass_a_f32(const BatchArgs& A, const BlockCounts& bc, bool nodal, cudaStream_t st);
int launch_pass_b_f32(const BatchArgs& A, const BlockCounts& bc, cudaStream_t st);
// Tile maps (tma::NMAP of them) of an FP32 slot; false if the slot cannot use tile loads.
bool encode_tile_maps(const SlotDesc& d, CUtensorMap* out);
bool tma_stencil_enabled();
int stencil_f32_occupancy(bool use_tma);

// process-wide count of kernels launched by the library
void count_launch(int n = 1);

// Stencil decomposition of one slot (tiles, z chunk, CTA counts): depends only on the
// slot's grid, so a slot's arithmetic is the same in any batch.
void decompose_slot(SlotDesc& d, int nodal);
constexpr int kMaxBlocksPerSlot = 4096;
// A slot's stencil decomposition takes the longest z chunk (64, 32, 16 or 8 planes) that still
// gives the slot alone this many CTAs per SM (152 SMs).
#ifndef TEM_SLOT_CTAS_PER_SM
#define TEM_SLOT_CTAS_PER_SM 2
#endif

// An FP32 inner solve whose recursive residual has not reached a new minimum for this many
// iterations ends, and the FP64 outer step restarts from the true residual.
#ifndef TEM_STALL_WINDOW
#define TEM_STALL_WINDOW 400
#endif

}  // namespace tem
