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
#include <cstring>

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
  while (d.zchunk > 8 && cols * ((d.g.nz + d.zchunk - 1) / d.zchunk) < 2 * 152) d.zchunk /= 2;
  d.zchunks = (d.g.nz + d.zchunk - 1) / d.zchunk;
  d.nblk_stencil = d.tiles_x * d.tiles_y * d.zchunks;
  const int64_t n = 3 * d.g.ncomp + (nodal ? d.g.ncomp : 0);
  d.nblk_update = (int)std::max<int64_t>(1, std::min<int64_t>(2048, (n + NT * 8 - 1) / (NT * 8)));
  d.nblk_nodal = (int)std::max<int64_t>(1, std::min<int64_t>(2048, (d.g.ncomp + NT * 8 - 1) / (NT * 8)));
}

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
  int blk_s = 0, blk_u = 0, blk_n = 0, max_part = 0;
  for (auto& d : slots_h_) {
    decompose_slot(d, nodal_);
    d.blk_stencil0 = blk_s;
    d.blk_update0 = blk_u;
    d.blk_nodal0 = blk_n;
    blk_s += d.nblk_stencil;
    blk_u += d.nblk_update;
    blk_n += d.nblk_nodal;
    max_part = std::max(max_part, std::max(d.nblk_stencil, std::max(d.nblk_update, d.nblk_nodal)) * 4);
  }
  nblk_stencil_ = blk_s;
  nblk_update_ = blk_u;
  nblk_nodal_ = blk_n;
  part_stride_ = max_part;
  std::vector<int> map(blk_s + blk_u + blk_n);
  for (int q = 0; q < ns; ++q) {
    const SlotDesc& d = slots_h_[q];
    for (int b = 0; b < d.nblk_stencil; ++b) map[d.blk_stencil0 + b] = q;
    for (int b = 0; b < d.nblk_update; ++b) map[blk_s + d.blk_update0 + b] = q;
    for (int b = 0; b < d.nblk_nodal; ++b) map[blk_s + blk_u + d.blk_nodal0 + b] = q;
  }
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
  TEM_TRY(map_d_.alloc(map.size() * sizeof(int), st));
  TEM_TRY(part_d_.alloc((size_t)ns * part_stride_ * sizeof(double), st));
  TEM_TRY(ticket_d_.alloc(ns * sizeof(unsigned), st));
  TEM_TRY(counters_d_.alloc(2 * sizeof(int), st));
  TEM_CUDA_TRY(cudaMemcpyAsync(slots_d_.ptr, slots_h_.data(), ns * sizeof(SlotDesc), cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemcpyAsync(sc_d_.ptr, sc_h_.data(), ns * sizeof(SlotScalars), cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemcpyAsync(map_d_.ptr, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, st));
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
                           const DevBuf& part, const DevBuf& ticket, const DevBuf& counters, int stride) {
  BatchArgs A;
  A.slots = slots.as<SlotDesc>();
  A.sc = sc.as<SlotScalars>();
  A.blk2slot = map.as<int>();
  A.ublk2slot = map.as<int>() + nblk_s;
  A.nblk2slot = map.as<int>() + nblk_s + nblk_u;
  A.part = part.as<double>();
  A.ticket = ticket.as<unsigned>();
  A.n_active = counters.as<int>();
  A.part_stride = stride;
  return A;
}

int Batch::launch_stencil(cudaStream_t st) {
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, nblk_stencil_, nblk_update_, part_d_, ticket_d_, counters_d_, part_stride_);
  if (precision_ == TEM_PREC_FP64) {
    k_cocg_stencil<double><<<nblk_stencil_, NT, 0, st>>>(A);
    TEM_CUDA_TRY(cudaGetLastError());
  } else {
    TEM_CUDA_TRY(launch_stencil_pipe(A, nblk_stencil_, st));
  }
  count_launch();
  return TEM_OK;
}

int Batch::launch_update(cudaStream_t st) {
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, nblk_stencil_, nblk_update_, part_d_, ticket_d_, counters_d_, part_stride_);
  if (precision_ == TEM_PREC_FP64)
    k_cocg_update<double><<<nblk_update_, NT, 0, st>>>(A);
  else
    k_cocg_update<float><<<nblk_update_, NT, 0, st>>>(A);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

int Batch::launch_nodal(cudaStream_t st, int init_only) {
  if (!nodal_) return TEM_OK;
  if (!init_only) return TEM_EINVAL;  // the per-iteration nodal work is inside passes A and B
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, nblk_stencil_, nblk_update_, part_d_, ticket_d_, counters_d_, part_stride_);
  if (precision_ == TEM_PREC_FP64)
    k_cocg_nodal<double, true><<<nblk_nodal_, NT, 0, st>>>(A);
  else
    k_cocg_nodal<float, true><<<nblk_nodal_, NT, 0, st>>>(A);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

int Batch::launch_iteration(cudaStream_t st) {
  TEM_TRY(launch_stencil(st));
  return launch_update(st);
}

int Batch::launches_per_iteration() const { return 2; }

int Batch::launch_residual(cudaStream_t st) {
  BatchArgs A = make_args(slots_d_, sc_d_, map_d_, nblk_stencil_, nblk_update_, part_d_, ticket_d_, counters_d_, part_stride_);
  int* n_done = counters_d_.as<int>() + 1;
  if (precision_ == TEM_PREC_FP64)
    k_residual<double><<<nblk_stencil_, NT, 0, st>>>(A, n_done);
  else
    k_residual<float><<<nblk_stencil_, NT, 0, st>>>(A, n_done);
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
    return TEM_OK;
  };
  TEM_TRY(launch_residual(st));
  TEM_TRY(launch_nodal(st, 1));
  launches += 2;
  TEM_TRY(poll());
  int64_t rounds = 0;
  while (counters_h_[1] < ns) {
    if (++rounds > max_rounds) return TEM_ETIMEOUT;
    if (counters_h_[0] > 0) {
      for (int it = 0; it < every; ++it) {
        TEM_TRY(launch_iteration(st));
        launches += launches_per_iteration();
      }
    }
    // slots whose inner solve ended take their FP64 outer step (the others skip it),
    // and the nodal pass starts the inner solves that step armed
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

int Batch::fetch_scalars(cudaStream_t st) {
  TEM_CUDA_TRY(cudaMemcpyAsync(sc_h_.data(), sc_d_.ptr, sc_h_.size() * sizeof(SlotScalars), cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  return TEM_OK;
}

}  // namespace tem
