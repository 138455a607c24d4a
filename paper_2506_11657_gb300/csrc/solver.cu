// Batched shifted COCG with FP64 defect correction (see kernels.cuh).
//
// Each slot solves (K - xi M) x = b.  Outer loop (FP64): r = b - A x; stop when
// ||r|| <= tol ||b||; otherwise run an inner Jacobi-COCG (van der Vorst &
// Melissen 1990, the unconjugated bilinear form for complex symmetric A):
//   FP64 mode : the inner iterate is x itself, aiming at tol/2 directly; the
//               outer step re-checks the true residual (residual replacement).
//   MIXED mode: the inner solve runs in FP32 on A d = s r (s ~ 1/||r||) to a
//               relative reduction inner_tol; the next outer step adds d / s
//               to x in FP64 and recomputes r in FP64 (defect correction).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "kernels.cuh"
#include "solver.h"

namespace tem {

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches += n; }
int64_t launch_count() { return g_launches.load(); }

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Per slot: x64[2] (FP64 edge vectors), then x, w, a0, a1, q (inner edge vectors) and
// xn, psi, b0, b1, cn, u, gp (inner nodal vectors) in the inner precision.
size_t slot_vector_bytes(int64_t ncomp, int precision) {
  const size_t es = precision == TEM_PREC_FP64 ? 16 : 8;
  const size_t v64 = align256(3 * (size_t)ncomp * 16);
  const size_t ve = align256(3 * (size_t)ncomp * es), vn = align256((size_t)ncomp * es);
  return 2 * v64 + 5 * ve + 7 * vn;
}

// Update-pass CTAs per slot: about TEM_UPD_PER_THREAD entries per thread, at most
// TEM_UPD_MAX_BLOCKS CTAs (a function of the slot's grid only, like every decomposition here).
// Each CTA first walks a chain of dependent loads (block list, slot scalars, descriptor) and ends
// with a block reduction, so it should stream several rounds of pairs in between.
#ifndef TEM_UPD_PER_THREAD
#define TEM_UPD_PER_THREAD 32
#endif
#ifndef TEM_UPD_MAX_BLOCKS
#define TEM_UPD_MAX_BLOCKS 512
#endif

SlotVectors carve_slot(void* base, int64_t ncomp, int precision) {
  const size_t es = precision == TEM_PREC_FP64 ? 16 : 8;
  const size_t v64 = align256(3 * (size_t)ncomp * 16);
  const size_t ve = align256(3 * (size_t)ncomp * es), vn = align256((size_t)ncomp * es);
  char* b = static_cast<char*>(base);
  SlotVectors v;
  v.x64[0] = b;
  v.x64[1] = b + v64;
  char* e = b + 2 * v64;
  v.x = e; v.w = e + ve; v.a0 = e + 2 * ve; v.a1 = e + 3 * ve; v.q = e + 4 * ve;
  char* n = e + 5 * ve;
  v.xn = n; v.psi = n + vn; v.b0 = n + 2 * vn; v.b1 = n + 3 * vn; v.cn = n + 4 * vn;
  v.u = n + 5 * vn; v.gp = n + 6 * vn;
  return v;
}

void decompose_slot(SlotDesc& d, int nodal) {
  d.tiles_x = (d.g.nx + TX - 1) / TX;
  d.tiles_y = (d.g.ny + TY - 1) / TY;
  // the longest z chunk (64/32/16/8 planes) that gives the slot alone 2 CTAs per SM (152 SMs)
  const int64_t cols = (int64_t)d.tiles_x * d.tiles_y;
  d.zchunk = ZMAX;
  while (d.zchunk > 8 && cols * ((d.g.nz + d.zchunk - 1) / d.zchunk) < TEM_SLOT_CTAS_PER_SM * 152) d.zchunk /= 2;
  d.zchunks = (d.g.nz + d.zchunk - 1) / d.zchunk;
  d.nblk_stencil = d.tiles_x * d.tiles_y * d.zchunks;
  const int64_t n = 3 * d.g.ncomp + (nodal ? d.g.ncomp : 0);
  d.nblk_update = (int)std::max<int64_t>(1, std::min<int64_t>(TEM_UPD_MAX_BLOCKS, (n + NT * TEM_UPD_PER_THREAD - 1) /
                                                                                    (NT * TEM_UPD_PER_THREAD)));
  d.nblk_nodal = (int)std::max<int64_t>(1, std::min<int64_t>(2048, (d.g.ncomp + NT * 8 - 1) / (NT * 8)));
}

// ---------------------------------------------------------------- block lists
// The CTAs of every used slot, interleaved by block index: block b of slot 0, of slot 1, ...,
// then block b+1.  Slots of one grid (the shifts of a model) then sweep the same tile at the same
// time, so the grid's shared arrays (masses, diag K) come from L2 for all but the first.  The
// stencil and update lists put the slots with d.tma first (their own launches).
void build_block_maps(const std::vector<SlotDesc>& slots, const std::vector<char>& use, std::vector<int2>& map,
                      BlockCounts* bc) {
  map.clear();
  const int ns = (int)slots.size();
  auto one = [&](auto nblk_of, int cls) {   // cls: 1 tma slots only, 0 the others, -1 all
    int most = 0;
    for (int q = 0; q < ns; ++q)
      if (use[q]) most = std::max(most, nblk_of(slots[q]));
    const size_t start = map.size();
    for (int b = 0; b < most; ++b)
      for (int q = 0; q < ns; ++q)
        if (use[q] && b < nblk_of(slots[q]) && (cls < 0 || (slots[q].tma != 0) == (cls == 1)))
          map.push_back(make_int2(q, b));
    return (int)(map.size() - start);
  };
  auto st = [](const SlotDesc& d) { return d.nblk_stencil; };
  auto up = [](const SlotDesc& d) { return d.nblk_update; };
  auto no = [](const SlotDesc& d) { return d.nblk_nodal; };
  bc->s_fast = one(st, 1);
  bc->s = bc->s_fast + one(st, 0);
  bc->u_fast = one(up, 1);
  bc->u = bc->u_fast + one(up, 0);
  bc->n = one(no, -1);
}

// ------------------------------------------------------------ TMA tile maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

static bool encode(EncodeTiledFn f, CUtensorMap* m, int rank, const void* base, const cuuint64_t* dim,
                   const cuuint64_t* stride, const cuuint32_t* box) {
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), dim, stride, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The seven tile maps of one FP32 slot (w, a0, a1, psi, b0, b1 and the packed masses), in the
// order of tma::MAP_*.  A complex FP32 vector is addressed as floats: x runs over 2 nx floats,
// so a box starting at column i0-2 starts at float 2 (i0-2), a multiple of 4 (16 bytes).
// Returns false when the layout does not allow tile loads (odd nx) or encoding fails.
bool encode_tile_maps(const SlotDesc& d, CUtensorMap* out) {
  const GridView& g = d.g;
  if (!tma_layout_ok(g) || !g.Mq) return false;
  EncodeTiledFn f = encode_fn();
  if (!f) return false;
  const cuuint64_t nx = g.nx, ny = g.ny, nz = g.nz;
  const cuuint64_t dv[4] = {2 * nx, ny, nz, 3}, sv[3] = {8 * nx, 8 * nx * ny, 8 * (cuuint64_t)g.ncomp};
  const cuuint32_t bv[4] = {2 * tma::BX, tma::BY, 1, 3};
  const cuuint64_t dn[3] = {2 * nx, ny, nz}, sn[2] = {8 * nx, 8 * nx * ny};
  const cuuint32_t bn[3] = {2 * tma::BX, tma::BY, 1};
  const cuuint64_t dm[4] = {4, nx, ny, nz}, sm[3] = {16, 16 * nx, 16 * nx * ny};
  const cuuint32_t bmq[4] = {4, tma::MX, tma::MY, 1};
  bool ok = encode(f, out + tma::MAP_W, 4, d.w, dv, sv, bv) && encode(f, out + tma::MAP_A0, 4, d.a0, dv, sv, bv) &&
            encode(f, out + tma::MAP_A1, 4, d.a1, dv, sv, bv) && encode(f, out + tma::MAP_PSI, 3, d.psi, dn, sn, bn) &&
            encode(f, out + tma::MAP_B0, 3, d.b0, dn, sn, bn) && encode(f, out + tma::MAP_B1, 3, d.b1, dn, sn, bn) &&
            encode(f, out + tma::MAP_MQ, 4, g.Mq, dm, sm, bmq);
  return ok;
}

// FP32 stencil kernel choice: the TMA kernel where every slot allows it, unless the environment
// variable TEM_FP32_STENCIL=pipe selects the cp.async kernel (for comparisons).
bool tma_stencil_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* v = std::getenv("TEM_FP32_STENCIL");
    on = (v && std::strcmp(v, "pipe") == 0) ? 0 : 1;
  }
  return on == 1;
}

int launch_pass_a_f32(const BatchArgs& A, const BlockCounts& bc, bool nodal, cudaStream_t st) {
  if (bc.s_fast > 0) {
    TEM_CUDA_TRY(launch_stencil_tma(A, bc.s_fast, nodal, st));
    count_launch();
  }
  if (bc.s > bc.s_fast) {
    BatchArgs B = A;
    B.blk2slot += bc.s_fast;
    TEM_CUDA_TRY(launch_stencil_pipe(B, bc.s - bc.s_fast, st));
    count_launch();
  }
  return TEM_OK;
}

int launch_pass_b_f32(const BatchArgs& A, const BlockCounts& bc, cudaStream_t st) {
  if (bc.u_fast > 0) {
    k_cocg_update_vec<<<bc.u_fast, NT, 0, st>>>(A);
    TEM_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  if (bc.u > bc.u_fast) {
    BatchArgs B = A;
    B.ublk2slot += bc.u_fast;
    k_cocg_update<float><<<bc.u - bc.u_fast, NT, 0, st>>>(B);
    TEM_CUDA_TRY(cudaGetLastError());
    count_launch();
  }
  return TEM_OK;
}

int stencil_f32_occupancy(bool use_tma) { return use_tma ? stencil_tma_occupancy() : stencil_pipe_occupancy(); }

Batch::~Batch() {
  if (counters_h_) cudaFreeHost(counters_h_);
}

int Batch::add_slot(const GridView& g, double xi_re, double xi_im, const SlotVectors& v,
                    const double* f_real, const void* rhs_complex, int rhs_div) {
  if ((int64_t)slots_h_.size() >= (1 << 20)) return TEM_EINVAL;
  SlotDesc d;
  std::memset(&d, 0, sizeof(d));
  d.g = g;
  d.xi_re = xi_re;
  d.xi_im = xi_im;
  d.x = v.x;
  d.w = v.w;
  d.a0 = v.a0;
  d.a1 = v.a1;
  d.q = v.q;
  d.xn = v.xn;
  d.psi = v.psi;
  d.b0 = v.b0;
  d.b1 = v.b1;
  d.cn = v.cn;
  d.u = v.u;
  d.gp = v.gp;
  d.x64[0] = v.x64[0];
  d.x64[1] = v.x64[1];
  d.f = f_real;
  d.rhs_c = static_cast<const double*>(rhs_complex);
  d.rhs_div = rhs_complex && rhs_div ? 1 : 0;
  d.fp64_inner = precision_ == TEM_PREC_FP64 ? 1 : 0;
  d.nodal = nodal_;
  d.div_nx = make_fastdiv((uint32_t)g.nx);
  d.div_ny = make_fastdiv((uint32_t)g.ny);
  d.div_nynz = make_fastdiv((uint32_t)(g.ny * g.nz));
  slots_h_.push_back(d);
  return TEM_OK;
}

int Batch::setup(const tem_options& opt, cudaStream_t st, const double* ff) {
  const int ns = (int)slots_h_.size();
  if (ns == 0) return TEM_EINVAL;
  int max_part = 0;
  for (auto& d : slots_h_) {
    decompose_slot(d, nodal_);
    max_part = std::max(max_part, std::max(d.nblk_stencil, std::max(d.nblk_update, d.nblk_nodal)) * 4);
  }
  part_stride_ = max_part;
  std::vector<int2> map;
  used_.assign(ns, 1);
  // tile maps of the FP32 stencil pass (slots that cannot use them take the cp.async kernel)
  std::vector<CUtensorMap> tm;
  const bool want_tma = precision_ == TEM_PREC_MIXED && tma_stencil_enabled();
  if (want_tma) {
    tm.resize((size_t)ns * tma::NMAP);
    for (int q = 0; q < ns; ++q)
      slots_h_[q].tma = encode_tile_maps(slots_h_[q], tm.data() + (size_t)q * tma::NMAP) ? 1 : 0;
  }
  build_block_maps(slots_h_, used_, map, &bc_);
  sc_h_.assign(ns, SlotScalars());
  for (int q = 0; q < ns; ++q) {
    SlotScalars& S = sc_h_[q];
    std::memset(&S, 0, sizeof(S));
    S.max_iter = opt.max_iter;
    S.ff = ff[q];
    S.tol_outer2 = opt.tol * opt.tol * ff[q];
    S.inner_rel2 = opt.inner_tol * opt.inner_tol;
    S.scale = 1.0 / std::sqrt(ff[q]);
    S.inv_scale_prev = 1.0;
    S.max_outer = opt.max_outer;
    S.stall_window = TEM_STALL_WINDOW;
    S.carry = opt.carry_direction != 0;
    S.stalled = 0;
    S.carry_ratio = 0.0;
  }
  TEM_TRY(slots_d_.alloc(ns * sizeof(SlotDesc), st));
  TEM_TRY(sc_d_.alloc(ns * sizeof(SlotScalars), st));
  TEM_TRY(map_d_.alloc(map.size() * sizeof(int2), st));
  if (want_tma) {
    TEM_TRY(tmaps_d_.alloc(tm.size() * sizeof(CUtensorMap), st));
    TEM_CUDA_TRY(cudaMemcpyAsync(tmaps_d_.ptr, tm.data(), tm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
  }
  TEM_TRY(part_d_.alloc((size_t)ns * part_stride_ * sizeof(double), st));
  TEM_TRY(ticket_d_.alloc(ns * sizeof(unsigned), st));
  TEM_TRY(counters_d_.alloc(2 * sizeof(int), st));
  TEM_CUDA_TRY(cudaMemcpyAsync(slots_d_.ptr, slots_h_.data(), ns * sizeof(SlotDesc), cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemcpyAsync(sc_d_.ptr, sc_h_.data(), ns * sizeof(SlotScalars), cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemcpyAsync(map_d_.ptr, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemsetAsync(ticket_d_.ptr, 0, ns * sizeof(unsigned), st));
  TEM_CUDA_TRY(cudaMemsetAsync(counters_d_.ptr, 0, 2 * sizeof(int), st));
  // zero every vector: boundary entries must read as 0 and are never written
  for (auto& d : slots_h_) {
    const size_t bytes = slot_vector_bytes(d.g.ncomp, precision_);
    TEM_CUDA_TRY(cudaMemsetAsync(d.x64[0], 0, bytes, st));
  }
  if (!counters_h_) TEM_CUDA_TRY(cudaHostAlloc(&counters_h_, 2 * sizeof(int), cudaHostAllocDefault));
  return TEM_OK;
}

static BatchArgs make_args(const DevBuf& slots, const DevBuf& sc, const DevBuf& map, int nblk_s, int nblk_u,
                           const DevBuf& part, const DevBuf& ticket, const DevBuf& counters, int stride,
                           const DevBuf& tmaps) {
  BatchArgs A;
  A.slots = slots.as<SlotDesc>();
  A.sc = sc.as<SlotScalars>();
  A.blk2slot = map.as<int2>();
  A.ublk2slot = map.as<int2>() + nblk_s;
  A.nblk2slot = map.as<int2>() + nblk_s + nblk_u;
  A.tmaps = tmaps.as<CUtensorMap>();
  A.part = part.as<double>();
  A.ticket = ticket.as<unsigned>();
  A.n_active = counters.as<int>();
  A.part_stride = stride;
  return A;
}

int Batch::launch_stencil(cudaStream_t st) {
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, bc_.s, bc_.u, part_d_, ticket_d_, counters_d_, part_stride_, tmaps_d_);
  if (precision_ == TEM_PREC_FP64) {
    k_cocg_stencil<double><<<bc_.s, NT, 0, st>>>(A);
    TEM_CUDA_TRY(cudaGetLastError());
    count_launch();
    return TEM_OK;
  }
  return launch_pass_a_f32(A, bc_, nodal_ != 0, st);
}

int Batch::launch_update(cudaStream_t st) {
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, bc_.s, bc_.u, part_d_, ticket_d_, counters_d_, part_stride_, tmaps_d_);
  if (precision_ == TEM_PREC_FP64) {
    k_cocg_update<double><<<bc_.u, NT, 0, st>>>(A);
    count_launch();
    TEM_CUDA_TRY(cudaGetLastError());
    return TEM_OK;
  }
  return launch_pass_b_f32(A, bc_, st);
}

int Batch::launch_nodal(cudaStream_t st, int init_only) {
  if (!nodal_) return TEM_OK;
  if (!init_only) return TEM_EINVAL;  // the per-iteration nodal work is inside passes A and B
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, bc_.s, bc_.u, part_d_, ticket_d_, counters_d_, part_stride_, tmaps_d_);
  if (precision_ == TEM_PREC_FP64)
    k_cocg_nodal<double, true><<<bc_.n, NT, 0, st>>>(A);
  else
    k_cocg_nodal<float, true><<<bc_.n, NT, 0, st>>>(A);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

int Batch::launch_iteration(cudaStream_t st) {
  TEM_TRY(launch_stencil(st));
  return launch_update(st);
}

int Batch::launches_per_iteration() const {
  if (precision_ == TEM_PREC_FP64) return 2;
  return (bc_.s_fast > 0) + (bc_.s > bc_.s_fast) + (bc_.u_fast > 0) + (bc_.u > bc_.u_fast);
}

int Batch::launch_residual(cudaStream_t st) {
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, bc_.s, bc_.u, part_d_, ticket_d_, counters_d_, part_stride_, tmaps_d_);
  int* n_done = counters_d_.as<int>() + 1;
  if (precision_ == TEM_PREC_FP64)
    k_residual<double><<<bc_.s, NT, 0, st>>>(A, n_done);
  else
    k_residual<float><<<bc_.s, NT, 0, st>>>(A, n_done);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

int Batch::solve(const tem_options& opt, cudaStream_t st, SolveStats* stats) {
  const int ns = (int)slots_h_.size();
  const int every = std::max(1, std::min(opt.check_every, 4096));
  // hard bound on the host loop: every slot can take max_iter inner iterations per
  // outer step and max_outer outer steps
  const int64_t max_rounds = (int64_t)(opt.max_outer + 2) * ((opt.max_iter + every - 1) / every + 2);
  int launches = 0, outer = 0;
  auto poll = [&]() -> int {
    TEM_CUDA_TRY(cudaMemcpyAsync(counters_h_, counters_d_.ptr, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    TEM_CUDA_TRY(cudaStreamSynchronize(st));
    if (const unsigned long long f = take_bounds_fault(st)) {   // only in the bounds-checked build
      char msg[128];
      snprintf(msg, sizeof(msg), "bounds check failed: site %llu, index %llu", f >> 48, f & 0xffffffffffffull);
      set_last_error(msg, __FILE__, __LINE__);
      return TEM_ECUDA;
    }
    return TEM_OK;
  };
  NvtxRange range("tem: batched shifted COCG");
  {
    NvtxRange r("tem: FP64 residual + start");
    TEM_TRY(launch_residual(st));
    TEM_TRY(launch_nodal(st, 1));
  }
  launches += 2;
  TEM_TRY(poll());
  int done_seen = 0;
  int64_t rounds = 0;
  while (counters_h_[1] < ns) {
    if (counters_h_[1] != done_seen) {
      // some slots finished: launch only the others from now on
      done_seen = counters_h_[1];
      TEM_TRY(drop_done_slots(st));
    }
    if (++rounds > max_rounds) return TEM_ETIMEOUT;
    if (counters_h_[0] > 0) {
      NvtxRange r("tem: COCG iterations (stencil + update passes)");
      for (int it = 0; it < every; ++it) {
        TEM_TRY(launch_iteration(st));
        launches += launches_per_iteration();
      }
    }
    // slots whose inner solve ended take their FP64 outer step (the others skip it),
    // and the nodal pass starts the inner solves that step armed
    NvtxRange r("tem: FP64 residual + start");
    TEM_TRY(launch_residual(st));
    TEM_TRY(launch_nodal(st, 1));
    launches += 2;
    TEM_TRY(poll());
  }
  TEM_TRY(fetch_scalars(st));
  for (auto& S : sc_h_) outer = std::max(outer, (int)S.outer);
  if (stats) {
    stats->launches += launches;
    stats->outer_steps += outer;
  }
  return TEM_OK;
}

// Rebuild the block lists without the slots that are done (after a poll: nothing in flight).
// A slot's blocks keep their block indices, so its arithmetic is unchanged.
int Batch::drop_done_slots(cudaStream_t st) {
  TEM_TRY(fetch_scalars(st));
  for (size_t q = 0; q < sc_h_.size(); ++q) used_[q] = sc_h_[q].done ? 0 : 1;
  std::vector<int2> map;
  build_block_maps(slots_h_, used_, map, &bc_);
  if (map.empty()) return TEM_OK;
  TEM_CUDA_TRY(cudaMemcpyAsync(map_d_.ptr, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  return TEM_OK;
}

int Batch::fetch_scalars(cudaStream_t st) {
  TEM_CUDA_TRY(cudaMemcpyAsync(sc_h_.data(), sc_d_.ptr, sc_h_.size() * sizeof(SlotScalars), cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  return TEM_OK;
}

}  // namespace tem
