// tem_forward, tem_adjoint, tem_apply_operator: the C ABI over the batched solver.
//
// Forward (Eq. (rmjQ)):  d[r, k] = sum_i Re(c[i, k] q_r^T (K - xi_i M)^{-1} f).
// Adjoint (Sec. 4):      grad[c] = sum_i Re(xi_i lambda_i^T (dM/dlog sigma_c) x_i),
//                        lambda_i = (K - xi_i M)^{-1} sum_r beta[i, r] q_r,
//                        beta[i, r] = sum_k c[i, k] g[r, k].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>

#include "kernels.cuh"
#include "solver.h"

namespace tem {
int64_t launch_count();
}

using namespace tem;

struct tem_state {
  const tem_grid* grid = nullptr;
  uint64_t sigma_gen = 0;                   // the grid's conductivity generation at the forward call
  tem_options opt;
  int s = 0, K = 0, n_rx = 0;
  std::vector<double> xi, c;                // host copies
  std::vector<int64_t> term_edge;
  std::vector<double> term_w;
  std::vector<int> term_off;
  DevBuf sol;                               // per-slot vectors of the forward solve
  std::unique_ptr<Batch> batch;             // forward batch (holds x_i)
  std::vector<int32_t> iters;
  std::vector<double> relres;
};

namespace {

int validate_poles(const double* xi, const double* c, int64_t s, int64_t K) {
  if (!xi || !c || s < 1 || s > 64 || K < 1 || K > 100000) return TEM_EINVAL;
  for (int64_t q = 0; q < 2 * s; ++q)
    if (!std::isfinite(xi[q])) return TEM_EINVAL;
  for (int64_t q = 0; q < 2 * s * K; ++q)
    if (!std::isfinite(c[q])) return TEM_EINVAL;
  for (int64_t q = 0; q < s; ++q)
    if (xi[2 * q] >= 0.0 && xi[2 * q + 1] == 0.0) return TEM_EINVAL;  // a real pole on [0, inf) makes A_i singular
  return TEM_OK;
}

int use_nodal(const tem_options& o) {
  if (o.precond == TEM_PRECOND_NODAL) return 1;
  if (o.precond == TEM_PRECOND_JACOBI) return 0;
  return 1;
}

int validate_options(const tem_options& o) {
  if (o.precond < TEM_PRECOND_AUTO || o.precond > TEM_PRECOND_NODAL) return TEM_EINVAL;
  if (o.precision != TEM_PREC_FP64 && o.precision != TEM_PREC_MIXED) return TEM_EINVAL;
  if (!(o.tol > 0.0 && o.tol < 1.0)) return TEM_EINVAL;
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return TEM_EINVAL;
  if (o.max_iter < 1 || o.max_outer < 1 || o.check_every < 1) return TEM_EINVAL;
  return TEM_OK;
}

// Solve (K - xi_i M) x_i = b_i for all shifts of one grid; returns the batch.
int solve_shifts(const tem_grid* g, const double* xi, int s, const tem_options& opt, cudaStream_t st,
                 const double* f_dev, const void* rhs_c_dev, const double* bnorm2, DevBuf& vec,
                 std::unique_ptr<Batch>& batch, SolveStats* stats, int rhs_div = 0) {
  const int64_t ncomp = g->v.ncomp;
  const size_t per = slot_vector_bytes(ncomp, opt.precision);
  TEM_TRY(vec.alloc(per * s, st));
  batch.reset(new Batch(opt.precision, use_nodal(opt)));
  for (int i = 0; i < s; ++i) {
    SlotVectors v = carve_slot(static_cast<char*>(vec.ptr) + per * i, ncomp, opt.precision);
    const void* rc = rhs_c_dev ? static_cast<const char*>(rhs_c_dev) + (size_t)i * 3 * ncomp * 16 : nullptr;
    TEM_TRY(batch->add_slot(g->v, xi[2 * i], xi[2 * i + 1], v, f_dev, rc, rhs_div));
  }
  TEM_TRY(batch->setup(opt, st, bnorm2));
  return batch->solve(opt, st, stats);
}

int collect_status(const Batch& b, std::vector<int32_t>& iters, std::vector<double>& relres) {
  int rc = TEM_OK;
  iters.clear();
  relres.clear();
  for (const auto& S : b.scalars()) {
    iters.push_back(S.total_iters);
    relres.push_back(S.ff > 0 ? std::sqrt(S.rr64 / S.ff) : 0.0);
    if (S.status == TEM_ETIMEOUT) rc = TEM_ETIMEOUT;   // a bounded device wait ran out
    else if (S.status == TEM_EBREAKDOWN && rc != TEM_ETIMEOUT) rc = TEM_EBREAKDOWN;
    else if (S.status == TEM_ENOCONV && rc == TEM_OK) rc = TEM_ENOCONV;
  }
  return rc;
}

}  // namespace

extern "C" {

int tem_forward(const tem_grid* grid, const double* loop_xy, int64_t n_vertices, double z_loop, double current,
                const double* rx_xyz, int64_t n_rx, const double* xi, const double* c, int64_t s, int64_t K,
                const tem_options* opt_in, void* cuda_stream, double* dbzdt_out, tem_state** state_out) {
  NvtxRange range("tem_forward");
  if (!grid || !dbzdt_out || !rx_xyz || n_rx < 1 || n_rx > 4096) return TEM_EINVAL;
  if (state_out) *state_out = nullptr;
  tem_options opt;
  tem_default_options(&opt);
  if (opt_in) opt = *opt_in;
  TEM_TRY(validate_options(opt));
  TEM_TRY(validate_poles(xi, c, s, K));
  if (opt.keep_state && !state_out) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TEM_CUDA_TRY(cudaSetDevice(grid->device));
  // source and receivers (sparse term lists, host)
  std::vector<Term> fterms;
  TEM_TRY(build_source(grid, loop_xy, n_vertices, z_loop, current, fterms));
  std::unique_ptr<tem_state> S(new tem_state());
  S->grid = grid;
  S->sigma_gen = grid->sigma_gen;
  S->opt = opt;
  S->s = int(s);
  S->K = int(K);
  S->n_rx = int(n_rx);
  S->xi.assign(xi, xi + 2 * s);
  S->c.assign(c, c + 2 * s * K);
  S->term_off.push_back(0);
  for (int64_t r = 0; r < n_rx; ++r) {
    std::vector<Term> q;
    TEM_TRY(build_receiver(grid, rx_xyz + 3 * r, q));
    for (auto& t : q) {
      S->term_edge.push_back(t.edge);
      S->term_w.push_back(t.w);
    }
    S->term_off.push_back((int)S->term_edge.size());
  }
  const int64_t ncomp = grid->v.ncomp;
  // device: f (real, dense), the term lists, c and the output
  DevBuf fbuf, misc;
  const size_t nt = S->term_edge.size();
  TEM_TRY(fbuf.alloc(3 * ncomp * sizeof(double), st));
  const size_t misc_bytes = 256 + fterms.size() * 16 + nt * 16 + (n_rx + 1) * 8 + 2 * s * K * 8 + n_rx * K * 8 + 4096;
  TEM_TRY(misc.alloc(misc_bytes, st));
  char* m = misc.as<char>();
  int64_t* d_fidx = reinterpret_cast<int64_t*>(m);
  double* d_fval = reinterpret_cast<double*>(d_fidx + fterms.size());
  int64_t* d_tedge = reinterpret_cast<int64_t*>(d_fval + fterms.size());
  double* d_tw = reinterpret_cast<double*>(d_tedge + nt);
  double* d_c = d_tw + nt;
  double* d_out = d_c + 2 * s * K;
  int* d_toff = reinterpret_cast<int*>(d_out + n_rx * K);
  {
    std::vector<int64_t> fi(fterms.size());
    std::vector<double> fv(fterms.size());
    double ff = 0.0;
    for (size_t q = 0; q < fterms.size(); ++q) {
      fi[q] = fterms[q].edge;
      fv[q] = fterms[q].w;
      ff += fv[q] * fv[q];
    }
    TEM_CUDA_TRY(cudaMemsetAsync(fbuf.ptr, 0, 3 * ncomp * sizeof(double), st));
    if (!fi.empty()) {
      TEM_CUDA_TRY(cudaMemcpyAsync(d_fidx, fi.data(), fi.size() * 8, cudaMemcpyHostToDevice, st));
      TEM_CUDA_TRY(cudaMemcpyAsync(d_fval, fv.data(), fv.size() * 8, cudaMemcpyHostToDevice, st));
    }
    if (nt) {
      TEM_CUDA_TRY(cudaMemcpyAsync(d_tedge, S->term_edge.data(), nt * 8, cudaMemcpyHostToDevice, st));
      TEM_CUDA_TRY(cudaMemcpyAsync(d_tw, S->term_w.data(), nt * 8, cudaMemcpyHostToDevice, st));
    }
    TEM_CUDA_TRY(cudaMemcpyAsync(d_toff, S->term_off.data(), (n_rx + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    TEM_CUDA_TRY(cudaMemcpyAsync(d_c, c, 2 * s * K * 8, cudaMemcpyHostToDevice, st));
    k_scatter<<<(int)((fi.size() + 255) / 256 + 1), 256, 0, st>>>(d_fidx, d_fval, (int64_t)fi.size(), fbuf.as<double>());
    count_launch();
    TEM_CUDA_TRY(cudaGetLastError());
    std::vector<double> ffs(s, ff);
    SolveStats stats;
    int rc = solve_shifts(grid, xi, int(s), opt, st, fbuf.as<double>(), nullptr, ffs.data(), S->sol, S->batch, &stats);
    if (rc != TEM_OK) return rc;
  }
  k_project_combine<<<(int)n_rx, 128, 0, st>>>(S->batch->slots_device(), S->batch->scalars_device(), int(s),
                                                 d_tedge, d_tw, d_toff, d_c, int(K), d_out, int(n_rx));
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  TEM_CUDA_TRY(cudaMemcpyAsync(dbzdt_out, d_out, n_rx * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  const int rc = collect_status(*S->batch, S->iters, S->relres);
  if (rc == TEM_EBREAKDOWN || rc == TEM_ETIMEOUT) return rc;
  if (opt.keep_state) *state_out = S.release();
  else if (state_out) *state_out = nullptr;
  return rc;
}

int tem_forward_sources(const tem_grid* grid, const double* loops_xy, const int64_t* vert_off, int64_t n_src,
                        const double* z_loops, const double* currents, const double* rx_xyz, int64_t n_rx,
                        const double* xi, const double* c, int64_t s, int64_t K, const tem_options* opt_in,
                        void* cuda_stream, double* dbzdt_out) {
  if (!grid || !loops_xy || !vert_off || !z_loops || !currents || !rx_xyz || !dbzdt_out) return TEM_EINVAL;
  if (n_src < 1 || n_src > 1024 || n_rx < 1 || n_rx > 4096) return TEM_EINVAL;
  tem_options opt;
  tem_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.keep_state) return TEM_EINVAL;
  TEM_TRY(validate_options(opt));
  TEM_TRY(validate_poles(xi, c, s, K));
  if (vert_off[0] != 0) return TEM_EINVAL;
  for (int64_t j = 0; j < n_src; ++j)
    if (vert_off[j + 1] - vert_off[j] < 3) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TEM_CUDA_TRY(cudaSetDevice(grid->device));
  // sources and receivers (sparse term lists, host); validated before any device work
  std::vector<std::vector<Term>> fterms(n_src);
  for (int64_t j = 0; j < n_src; ++j)
    TEM_TRY(build_source(grid, loops_xy + 2 * vert_off[j], vert_off[j + 1] - vert_off[j], z_loops[j], currents[j],
                         fterms[j]));
  std::vector<int64_t> term_edge;
  std::vector<double> term_w;
  std::vector<int> term_off(1, 0);
  for (int64_t r = 0; r < n_rx; ++r) {
    std::vector<Term> q;
    TEM_TRY(build_receiver(grid, rx_xyz + 3 * r, q));
    for (auto& t : q) {
      term_edge.push_back(t.edge);
      term_w.push_back(t.w);
    }
    term_off.push_back((int)term_edge.size());
  }
  const int64_t ncomp = grid->v.ncomp;
  const size_t nt = term_edge.size();
  // one dense real source vector per loop
  DevBuf fbuf, misc, vec;
  TEM_TRY(fbuf.alloc((size_t)n_src * 3 * ncomp * sizeof(double), st));
  TEM_CUDA_TRY(cudaMemsetAsync(fbuf.ptr, 0, (size_t)n_src * 3 * ncomp * sizeof(double), st));
  size_t nf = 0;
  for (auto& ft : fterms) nf += ft.size();
  const size_t misc_bytes = 256 + nf * 16 + nt * 16 + (n_rx + 1) * 8 + 2 * s * K * 8 + (size_t)n_src * n_rx * K * 8;
  TEM_TRY(misc.alloc(misc_bytes, st));
  int64_t* d_fidx = misc.as<int64_t>();
  double* d_fval = reinterpret_cast<double*>(d_fidx + nf);
  int64_t* d_tedge = reinterpret_cast<int64_t*>(d_fval + nf);
  double* d_tw = reinterpret_cast<double*>(d_tedge + nt);
  double* d_c = d_tw + nt;
  double* d_out = d_c + 2 * s * K;
  int* d_toff = reinterpret_cast<int*>(d_out + (size_t)n_src * n_rx * K);
  std::vector<double> ffs;
  {
    std::vector<int64_t> fi;
    std::vector<double> fv;
    for (int64_t j = 0; j < n_src; ++j) {
      double ff = 0.0;
      for (auto& t : fterms[j]) {
        fi.push_back(j * 3 * ncomp + t.edge);
        fv.push_back(t.w);
        ff += t.w * t.w;
      }
      for (int64_t i = 0; i < s; ++i) ffs.push_back(ff);
    }
    if (!fi.empty()) {
      TEM_CUDA_TRY(cudaMemcpyAsync(d_fidx, fi.data(), fi.size() * 8, cudaMemcpyHostToDevice, st));
      TEM_CUDA_TRY(cudaMemcpyAsync(d_fval, fv.data(), fv.size() * 8, cudaMemcpyHostToDevice, st));
      k_scatter<<<(int)((fi.size() + 255) / 256 + 1), 256, 0, st>>>(d_fidx, d_fval, (int64_t)fi.size(),
                                                                     fbuf.as<double>());
      count_launch();
      TEM_CUDA_TRY(cudaGetLastError());
    }
    if (nt) {
      TEM_CUDA_TRY(cudaMemcpyAsync(d_tedge, term_edge.data(), nt * 8, cudaMemcpyHostToDevice, st));
      TEM_CUDA_TRY(cudaMemcpyAsync(d_tw, term_w.data(), nt * 8, cudaMemcpyHostToDevice, st));
    }
    TEM_CUDA_TRY(cudaMemcpyAsync(d_toff, term_off.data(), (n_rx + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    TEM_CUDA_TRY(cudaMemcpyAsync(d_c, c, 2 * s * K * 8, cudaMemcpyHostToDevice, st));
  }
  // all n_src * s systems in one batch: slot j * s + i is source j, shift i
  const size_t per = slot_vector_bytes(ncomp, opt.precision);
  TEM_TRY(vec.alloc(per * n_src * s, st));
  Batch b(opt.precision, use_nodal(opt));
  for (int64_t j = 0; j < n_src; ++j)
    for (int64_t i = 0; i < s; ++i)
      TEM_TRY(b.add_slot(grid->v, xi[2 * i], xi[2 * i + 1],
                         carve_slot(vec.as<char>() + per * (j * s + i), ncomp, opt.precision),
                         fbuf.as<double>() + j * 3 * ncomp, nullptr));
  TEM_TRY(b.setup(opt, st, ffs.data()));
  SolveStats stats;
  TEM_TRY(b.solve(opt, st, &stats));
  for (int64_t j = 0; j < n_src; ++j) {
    k_project_combine<<<(int)n_rx, 128, 0, st>>>(b.slots_device() + j * s, b.scalars_device() + j * s, int(s),
                                                   d_tedge, d_tw, d_toff, d_c, int(K), d_out + j * n_rx * K,
                                                   int(n_rx));
    count_launch();
    TEM_CUDA_TRY(cudaGetLastError());
  }
  TEM_CUDA_TRY(cudaMemcpyAsync(dbzdt_out, d_out, (size_t)n_src * n_rx * K * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int32_t> it;
  std::vector<double> rr;
  return collect_status(b, it, rr);
}

int tem_state_stats(const tem_state* state, int32_t* iters, double* relres) {
  if (!state) return TEM_EINVAL;
  for (int i = 0; i < state->s; ++i) {
    if (iters) iters[i] = state->iters[i];
    if (relres) relres[i] = state->relres[i];
  }
  return TEM_OK;
}

int tem_state_solution(const tem_state* state, int64_t i, void* cuda_stream, double* x_out) {
  if (!state || !x_out || !state->batch || i < 0 || i >= state->s) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const SlotDesc& d = state->batch->slots_host()[i];
  const SlotScalars& S = state->batch->scalars()[i];
  const size_t bytes = (size_t)3 * state->grid->v.ncomp * 16;
  TEM_CUDA_TRY(cudaMemcpyAsync(x_out, d.x64[S.xcur], bytes, cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  return TEM_OK;
}

int tem_state_fields(const tem_state* state, int64_t k0, int64_t nk, void* cuda_stream, void* u_dev) {
  if (!state || !u_dev || !state->batch || k0 < 0 || nk < 1 || k0 + nk > state->K) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TEM_CUDA_TRY(cudaSetDevice(state->grid->device));
  DevBuf cb;
  TEM_TRY(cb.alloc(state->c.size() * sizeof(double), st));
  TEM_CUDA_TRY(cudaMemcpyAsync(cb.ptr, state->c.data(), state->c.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  const int64_t n3 = 3 * state->grid->v.ncomp;
  const int64_t nblk = ((n3 + NT - 1) / NT) * nk;
  if (nblk > 2147483647LL) return TEM_EINVAL;
  k_fields<<<(unsigned)nblk, NT, 0, st>>>(state->batch->slots_device(), state->batch->scalars_device(), state->s,
                                     cb.as<double>(), state->K, int(k0), int(nk), n3, static_cast<double*>(u_dev));
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

int tem_adjoint(tem_state* S, const double* g, void* cuda_stream, double* grad) {
  NvtxRange range("tem_adjoint");
  if (!S || !g || !grad || !S->batch) return TEM_EINVAL;
  if (S->grid->sigma_gen != S->sigma_gen) {
    set_last_error("tem_adjoint: the grid's conductivity changed after the forward call", __FILE__, __LINE__);
    return TEM_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  for (int64_t q = 0; q < (int64_t)S->n_rx * S->K; ++q)
    if (!std::isfinite(g[q])) return TEM_EINVAL;
  const tem_grid* grid = S->grid;
  const int64_t ncomp = grid->v.ncomp;
  const int s = S->s, K = S->K, n_rx = S->n_rx;
  // beta[i, r] = sum_k c[i, k] g[r, k];  w_i = sum_r beta[i, r] q_r (unique edges per slot)
  std::vector<std::vector<std::pair<int64_t, std::pair<double, double>>>> w(s);
  std::vector<double> ww(s, 0.0);
  for (int i = 0; i < s; ++i) {
    std::map<int64_t, std::pair<double, double>> acc;
    for (int r = 0; r < n_rx; ++r) {
      double br = 0.0, bi = 0.0;
      for (int k = 0; k < K; ++k) {
        br += S->c[2 * (i * K + k)] * g[r * K + k];
        bi += S->c[2 * (i * K + k) + 1] * g[r * K + k];
      }
      for (int t = S->term_off[r]; t < S->term_off[r + 1]; ++t) {
        auto& a = acc[S->term_edge[t]];
        a.first += br * S->term_w[t];
        a.second += bi * S->term_w[t];
      }
    }
    for (auto& kv : acc) {
      w[i].push_back({kv.first, kv.second});
      ww[i] += kv.second.first * kv.second.first + kv.second.second * kv.second.second;
    }
  }
  bool all_zero = true;
  for (int i = 0; i < s; ++i) all_zero = all_zero && ww[i] == 0.0;
  if (all_zero) {
    std::memset(grad, 0, ncomp * sizeof(double));
    return TEM_OK;
  }
  for (int i = 0; i < s; ++i)
    if (ww[i] == 0.0) ww[i] = 1e-300;  // solve of a zero right-hand side ends at once
  DevBuf rhs, vec;
  TEM_TRY(rhs.alloc((size_t)s * 3 * ncomp * 16, st));
  TEM_CUDA_TRY(cudaMemsetAsync(rhs.ptr, 0, (size_t)s * 3 * ncomp * 16, st));
  {
    std::vector<int64_t> idx;
    std::vector<double> val;
    for (int i = 0; i < s; ++i)
      for (auto& e : w[i]) {
        idx.push_back((int64_t)i * 3 * ncomp + e.first);
        val.push_back(e.second.first);
        val.push_back(e.second.second);
      }
    DevBuf tmp;
    TEM_TRY(tmp.alloc(idx.size() * 8 + val.size() * 8 + 256, st));
    int64_t* d_idx = tmp.as<int64_t>();
    double* d_val = reinterpret_cast<double*>(d_idx + idx.size());
    TEM_CUDA_TRY(cudaMemcpyAsync(d_idx, idx.data(), idx.size() * 8, cudaMemcpyHostToDevice, st));
    TEM_CUDA_TRY(cudaMemcpyAsync(d_val, val.data(), val.size() * 8, cudaMemcpyHostToDevice, st));
    k_scatter_c<<<(int)((idx.size() + 255) / 256 + 1), 256, 0, st>>>(d_idx, d_val, (int64_t)idx.size(), rhs.as<double>());
    count_launch();
    TEM_CUDA_TRY(cudaGetLastError());
    TEM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  std::unique_ptr<Batch> ab;
  SolveStats stats;
  int rc = solve_shifts(grid, S->xi.data(), s, S->opt, st, nullptr, rhs.ptr, ww.data(), vec, ab, &stats);
  if (rc != TEM_OK) return rc;
  DevBuf gbuf;
  TEM_TRY(gbuf.alloc(ncomp * sizeof(double), st));
  k_gradient<<<152 * 8, 256, 0, st>>>(grid->v, grid->sig.as<double>(), S->batch->slots_device(),
                                       S->batch->scalars_device(), ab->slots_device(), ab->scalars_device(), s,
                                       gbuf.as<double>());
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  TEM_CUDA_TRY(cudaMemcpyAsync(grad, gbuf.ptr, ncomp * sizeof(double), cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int32_t> it;
  std::vector<double> rr;
  return collect_status(*ab, it, rr);
}

int tem_jvp(tem_state* S, const double* dlogsigma, void* cuda_stream, double* ddbzdt_out) {
  NvtxRange range("tem_jvp");
  if (!S || !dlogsigma || !ddbzdt_out || !S->batch) return TEM_EINVAL;
  if (S->grid->sigma_gen != S->sigma_gen) {
    set_last_error("tem_jvp: the grid's conductivity changed after the forward call", __FILE__, __LINE__);
    return TEM_EINVAL;
  }
  const tem_grid* grid = S->grid;
  const int64_t ncomp = grid->v.ncomp;
  bool any = false;
  for (int64_t q = 0; q < ncomp; ++q) {
    if (!std::isfinite(dlogsigma[q])) return TEM_EINVAL;
    any = any || dlogsigma[q] != 0.0;
  }
  const int s = S->s, K = S->K, n_rx = S->n_rx;
  if (!any) {
    std::memset(ddbzdt_out, 0, (size_t)n_rx * K * sizeof(double));
    return TEM_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TEM_CUDA_TRY(cudaSetDevice(grid->device));
  // right-hand sides b_i = xi_i dM x_i and their norms (fixed-order partial sums)
  DevBuf dmb, rhs, part;
  TEM_TRY(dmb.alloc(ncomp * sizeof(double), st));
  TEM_TRY(rhs.alloc((size_t)s * 3 * ncomp * 16, st));
  const int nb = 2 * 152;
  TEM_TRY(part.alloc((size_t)s * nb * sizeof(double), st));
  TEM_CUDA_TRY(cudaMemcpyAsync(dmb.ptr, dlogsigma, ncomp * sizeof(double), cudaMemcpyHostToDevice, st));
  k_jvp_rhs<<<152 * 8, 256, 0, st>>>(grid->v, grid->sig.as<double>(), dmb.as<double>(), S->batch->slots_device(),
                                      S->batch->scalars_device(), s, rhs.as<double>());
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  k_rhs_norm2<<<dim3(nb, s), NT, 0, st>>>(rhs.as<double>(), 3 * ncomp, part.as<double>());
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  std::vector<double> ph((size_t)s * nb), ww(s, 0.0);
  TEM_CUDA_TRY(cudaMemcpyAsync(ph.data(), part.ptr, ph.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < s; ++i) {
    for (int b = 0; b < nb; ++b) ww[i] += ph[(size_t)i * nb + b];
    if (ww[i] == 0.0) ww[i] = 1e-300;  // solve of a zero right-hand side ends at once
  }
  // the batched solves A_i dx_i = b_i (G^T b_i != 0 in general)
  DevBuf vec;
  std::unique_ptr<Batch> jb;
  SolveStats stats;
  int rc = solve_shifts(grid, S->xi.data(), s, S->opt, st, nullptr, rhs.ptr, ww.data(), vec, jb, &stats, 1);
  if (rc != TEM_OK) return rc;
  // dd[r, k] = sum_i Re(c_ik q_r^T dx_i)
  const size_t nt = S->term_edge.size();
  DevBuf misc;
  TEM_TRY(misc.alloc(256 + nt * 16 + (n_rx + 1) * 8 + 2 * (size_t)s * K * 8 + (size_t)n_rx * K * 8, st));
  int64_t* d_tedge = misc.as<int64_t>();
  double* d_tw = reinterpret_cast<double*>(d_tedge + nt);
  double* d_c = d_tw + nt;
  double* d_out = d_c + 2 * s * K;
  int* d_toff = reinterpret_cast<int*>(d_out + n_rx * K);
  if (nt) {
    TEM_CUDA_TRY(cudaMemcpyAsync(d_tedge, S->term_edge.data(), nt * 8, cudaMemcpyHostToDevice, st));
    TEM_CUDA_TRY(cudaMemcpyAsync(d_tw, S->term_w.data(), nt * 8, cudaMemcpyHostToDevice, st));
  }
  TEM_CUDA_TRY(cudaMemcpyAsync(d_toff, S->term_off.data(), (n_rx + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemcpyAsync(d_c, S->c.data(), 2 * (size_t)s * K * 8, cudaMemcpyHostToDevice, st));
  k_project_combine<<<n_rx, 128, 0, st>>>(jb->slots_device(), jb->scalars_device(), s, d_tedge, d_tw, d_toff, d_c, K,
                                           d_out, n_rx);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  TEM_CUDA_TRY(cudaMemcpyAsync(ddbzdt_out, d_out, (size_t)n_rx * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int32_t> it;
  std::vector<double> rr;
  return collect_status(*jb, it, rr);
}

int tem_state_destroy(tem_state* state) {
  if (!state) return TEM_EINVAL;
  cudaStreamSynchronize(state->sol.stream);
  delete state;
  return TEM_OK;
}

int tem_apply_operator(const tem_grid* grid, const double* xi, int64_t s, const void* p_dev, void* q_dev,
                       int32_t precision, void* cuda_stream) {
  if (!grid || !xi || !p_dev || !q_dev || s < 1 || s > 65535) return TEM_EINVAL;
  if (precision != TEM_PREC_FP64 && precision != TEM_PREC_MIXED) return TEM_EINVAL;
  for (int64_t q = 0; q < 2 * s; ++q)
    if (!std::isfinite(xi[q])) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  DevBuf dxi;
  TEM_TRY(dxi.alloc(2 * s * sizeof(double), st));
  TEM_CUDA_TRY(cudaMemcpyAsync(dxi.ptr, xi, 2 * s * sizeof(double), cudaMemcpyHostToDevice, st));
  const GridView& g = grid->v;
  const int zchunk = 32;
  const int tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY, tz = (g.nz + zchunk - 1) / zchunk;
  dim3 grd(tx * ty * tz, (unsigned)s);
  if (precision == TEM_PREC_FP64)
    k_apply<double><<<grd, NT, 0, st>>>(g, dxi.as<double>(), p_dev, q_dev, tx, ty, zchunk);
  else
    k_apply<float><<<grd, NT, 0, st>>>(g, dxi.as<double>(), p_dev, q_dev, tx, ty, zchunk);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

int64_t tem_launch_count(void) { return tem::launch_count(); }

int tem_profile_passes(const tem_grid* grid, const double* loop_xy, int64_t n_vertices, double z_loop,
                       double current, const double* xi, int64_t s, int32_t precision, int32_t precond,
                       int32_t n_iter,
                       void* cuda_stream, double* ms_out, double* units_out) {
  if (!grid || !xi || !ms_out || s < 1 || s > 64 || n_iter < 1 || n_iter > 100000) return TEM_EINVAL;
  if (precision != TEM_PREC_FP64 && precision != TEM_PREC_MIXED) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<Term> fterms;
  TEM_TRY(build_source(grid, loop_xy, n_vertices, z_loop, current, fterms));
  const int64_t ncomp = grid->v.ncomp;
  DevBuf fbuf, tbuf, vec;
  TEM_TRY(fbuf.alloc(3 * ncomp * sizeof(double), st));
  TEM_TRY(tbuf.alloc(fterms.size() * 16 + 256, st));
  std::vector<int64_t> fi;
  std::vector<double> fv;
  double ff = 0;
  for (auto& t : fterms) { fi.push_back(t.edge); fv.push_back(t.w); ff += t.w * t.w; }
  int64_t* d_fidx = tbuf.as<int64_t>();
  double* d_fval = reinterpret_cast<double*>(d_fidx + fi.size());
  TEM_CUDA_TRY(cudaMemsetAsync(fbuf.ptr, 0, 3 * ncomp * sizeof(double), st));
  TEM_CUDA_TRY(cudaMemcpyAsync(d_fidx, fi.data(), fi.size() * 8, cudaMemcpyHostToDevice, st));
  TEM_CUDA_TRY(cudaMemcpyAsync(d_fval, fv.data(), fv.size() * 8, cudaMemcpyHostToDevice, st));
  k_scatter<<<(int)((fi.size() + 255) / 256 + 1), 256, 0, st>>>(d_fidx, d_fval, (int64_t)fi.size(), fbuf.as<double>());
  count_launch();
  tem_options opt;
  tem_default_options(&opt);
  opt.precision = precision;
  opt.precond = precond;
  if (validate_options(opt) != TEM_OK) return TEM_EINVAL;
  opt.tol = 1e-300;   // nothing converges during the timed iterations
  opt.inner_tol = 1e-300;
  const size_t per = slot_vector_bytes(ncomp, precision);
  TEM_TRY(vec.alloc(per * s, st));
  Batch b(precision, use_nodal(opt));
  for (int i = 0; i < s; ++i)
    TEM_TRY(b.add_slot(grid->v, xi[2 * i], xi[2 * i + 1], carve_slot(vec.as<char>() + per * i, ncomp, precision),
                       fbuf.as<double>(), nullptr));
  std::vector<double> ffs(s, ff);
  TEM_TRY(b.setup(opt, st, ffs.data()));
  cudaEvent_t ev[2];
  TEM_CUDA_TRY(cudaEventCreate(&ev[0]));
  TEM_CUDA_TRY(cudaEventCreate(&ev[1]));
  float ms = 0;
  TEM_CUDA_TRY(cudaEventRecord(ev[0], st));
  TEM_TRY(b.launch_residual(st));
  TEM_CUDA_TRY(cudaEventRecord(ev[1], st));
  TEM_CUDA_TRY(cudaEventSynchronize(ev[1]));
  TEM_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
  ms_out[2] = ms;
  TEM_TRY(b.launch_nodal(st, 1));
  double tot_s = 0, tot_u = 0;
  for (int it = 0; it < n_iter; ++it) {
    TEM_CUDA_TRY(cudaEventRecord(ev[0], st));
    TEM_TRY(b.launch_stencil(st));
    TEM_CUDA_TRY(cudaEventRecord(ev[1], st));
    TEM_CUDA_TRY(cudaEventSynchronize(ev[1]));
    TEM_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    tot_s += ms;
    TEM_CUDA_TRY(cudaEventRecord(ev[0], st));
    TEM_TRY(b.launch_update(st));
    TEM_CUDA_TRY(cudaEventRecord(ev[1], st));
    TEM_CUDA_TRY(cudaEventSynchronize(ev[1]));
    TEM_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    tot_u += ms;
  }
  ms_out[0] = tot_s / n_iter;
  ms_out[1] = tot_u / n_iter;
  ms_out[3] = precision == TEM_PREC_MIXED ? stencil_f32_occupancy(b.uses_tma()) : 0;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (units_out) {
    const int64_t nx = grid->v.nx, ny = grid->v.ny, nz = grid->v.nz;
    const int64_t interior = nx * (ny - 1) * (nz - 1) + (nx - 1) * ny * (nz - 1) + (nx - 1) * (ny - 1) * nz;
    units_out[0] = double(interior) * double(s);
  }
  TEM_TRY(b.fetch_scalars(st));
  for (const auto& S : b.scalars())
    if (S.status != TEM_OK || !S.active) return TEM_EBREAKDOWN;  // a slot stopped: the timing is not of s slots
  return TEM_OK;
}

}  // extern "C"

// ------------------------------------------------ the single-time baseline (Sec. 3.1)
extern "C" int tem_forward_single_time(const tem_grid* grid, const double* loop_xy, int64_t n_vertices, double z_loop,
                                       double current, const double* rx_xyz, int64_t n_rx, const double* t, int64_t K,
                                       const double* xi, const double* c, int64_t s, const tem_options* opt_in,
                                       void* cuda_stream, double* dbzdt_out, int64_t* solves_out) {
  NvtxRange range("tem_forward_single_time");
  if (!grid || !t || !dbzdt_out || !rx_xyz || K < 1 || K > 100000 || n_rx < 1 || n_rx > 4096) return TEM_EINVAL;
  TEM_TRY(validate_poles(xi, c, s, 1));
  for (int64_t k = 0; k < K; ++k)
    if (!(std::isfinite(t[k]) && t[k] > 0.0)) return TEM_EINVAL;
  tem_options opt;
  tem_default_options(&opt);
  if (opt_in) opt = *opt_in;
  opt.keep_state = 0;
  // channel k takes its own s systems (t_k K - xi_i M) x = f, i.e. the shifts xi_i / t_k with
  // the weights c_i / t_k on channel k alone; they go through the batched solver 64 at a time
  const int64_t total = s * K;
  std::vector<double> sum((size_t)n_rx * K, 0.0), part((size_t)n_rx * K);
  int worst = TEM_OK;
  for (int64_t j0 = 0; j0 < total; j0 += 64) {
    const int64_t ns = std::min<int64_t>(64, total - j0);
    std::vector<double> xs(2 * ns), cs(2 * ns * K, 0.0);
    for (int64_t j = 0; j < ns; ++j) {
      const int64_t q = j0 + j, k = q / s, i = q % s;
      xs[2 * j] = xi[2 * i] / t[k];
      xs[2 * j + 1] = xi[2 * i + 1] / t[k];
      cs[2 * (j * K + k)] = c[2 * i] / t[k];
      cs[2 * (j * K + k) + 1] = c[2 * i + 1] / t[k];
    }
    const int rc = tem_forward(grid, loop_xy, n_vertices, z_loop, current, rx_xyz, n_rx, xs.data(), cs.data(), ns, K,
                               &opt, cuda_stream, part.data(), nullptr);
    if (rc != TEM_OK && rc != TEM_ENOCONV) return rc;
    if (rc == TEM_ENOCONV) worst = TEM_ENOCONV;
    for (size_t q = 0; q < sum.size(); ++q) sum[q] += part[q];
  }
  std::memcpy(dbzdt_out, sum.data(), sum.size() * sizeof(double));
  if (solves_out) *solves_out = total;
  return worst;
}
