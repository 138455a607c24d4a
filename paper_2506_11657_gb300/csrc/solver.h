// Batched shifted COCG driver: many (problem, shift) slots advanced together.
#pragma once

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

  int stencil_blocks() const { return nblk_stencil_; }
  int update_blocks() const { return nblk_update_; }
  int nodal_blocks() const { return nblk_nodal_; }
  // launch one (stencil, update) pair or one residual pass for all slots (bench / profiling)
  int launch_iteration(cudaStream_t st);
  int launches_per_iteration() const;
  int launch_stencil(cudaStream_t st);
  int launch_update(cudaStream_t st);
  int launch_nodal(cudaStream_t st, int init_only);
  int launch_residual(cudaStream_t st);

 private:
  int precision_;
  int nodal_;
  std::vector<SlotDesc> slots_h_;
  std::vector<SlotScalars> sc_h_;
  int nblk_stencil_ = 0, nblk_update_ = 0, nblk_nodal_ = 0;
  int part_stride_ = 0;
  DevBuf slots_d_, sc_d_, map_d_, part_d_, ticket_d_, counters_d_;
  int* counters_h_ = nullptr;   // pinned: [n_active, n_done]
};

// process-wide count of kernels launched by the library
void count_launch(int n = 1);

// Stencil decomposition of one slot (tiles, z chunk, CTA counts): depends only on the
// slot's grid, so a slot's arithmetic is the same in any batch.
void decompose_slot(SlotDesc& d, int nodal);
constexpr int kMaxBlocksPerSlot = 4096;

// An FP32 inner solve whose recursive residual has not reached a new minimum for this many
// iterations ends, and the FP64 outer step restarts from the true residual.
#ifndef TEM_STALL_WINDOW
#define TEM_STALL_WINDOW 400
#endif

}  // namespace tem
