// Continuous batching of forward models (see the serving section of tem.h).
//
// The server keeps one table of slots (one slot = one shifted system) in device
// memory.  A request takes a contiguous range of slots for its shifts while it runs.
// Every step launches the same passes as a single forward solve -- FP64 residual and
// nodal start for the slots between inner solves, then iters_per_step rounds of the
// stencil, update and nodal passes -- over the block lists of all running slots.
// Slots keep their own tiling (decompose_slot) and reduce only over their own blocks,
// so a request's arithmetic does not depend on what else runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>

#include "kernels.cuh"
#include "solver.h"

using namespace tem;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t ticket = 0;
  std::vector<double> hx, hy, hz, sigma, loop, rx, xi, c;
  double origin[3] = {0, 0, 0};
  double z_loop = 0, current = 1;
  int s = 0, K = 0, n_rx = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int first_slot = -1;
  size_t footprint = 0;
  tem_grid* grid = nullptr;
  DevBuf fbuf, vec, misc;
  int64_t* d_tedge = nullptr;
  double* d_tw = nullptr;
  int* d_toff = nullptr;
  double* d_c = nullptr;
  double* d_out = nullptr;
  std::vector<double> d;
  int status = TEM_OK;
  int max_iters = 0;
  ~Request() {
    fbuf.release();
    vec.release();
    misc.release();
    if (grid) tem_grid_destroy(grid);
  }
};

// A host-only grid stub for validating geometry at submit time (no device memory).
struct HostGrid {
  tem_grid g;
  HostGrid(const Request& r) {
    g.hx = r.hx;
    g.hy = r.hy;
    g.hz = r.hz;
    for (int q = 0; q < 3; ++q) g.origin[q] = r.origin[q];
    g.v.nx = (int)r.hx.size();
    g.v.ny = (int)r.hy.size();
    g.v.nz = (int)r.hz.size();
    g.v.ncomp = (int64_t)g.v.nx * g.v.ny * g.v.nz;
  }
};

bool all_finite_positive(const double* a, int64_t n) {
  for (int64_t q = 0; q < n; ++q)
    if (!(std::isfinite(a[q]) && a[q] > 0)) return false;
  return true;
}

}  // namespace

struct tem_server {
  tem_server_options opt;
  cudaStream_t st = nullptr;
  int nodal = 1;
  std::vector<SlotDesc> slots_h;
  std::vector<SlotScalars> sc_h;
  std::vector<int> owner;  // request ticket per slot, -1 when free
  DevBuf slots_d, sc_d, part_d, ticket_d, counters_d, map_d, tmaps_d;
  BlockCounts bc;               // sizes of the block lists
  std::vector<char> in_maps;   // slots in the current block lists
  int part_stride = 4 * kMaxBlocksPerSlot;
  bool maps_dirty = true;
  std::deque<std::unique_ptr<Request>> queue;
  std::vector<std::unique_ptr<Request>> running;
  std::map<int64_t, std::unique_ptr<Request>> finished;
  size_t used = 0;
  int64_t next_ticket = 1;

  BatchArgs args() const {
    BatchArgs A;
    A.slots = slots_d.as<SlotDesc>();
    A.sc = sc_d.as<SlotScalars>();
    A.blk2slot = map_d.as<int2>();
    A.ublk2slot = map_d.as<int2>() + bc.s;
    A.nblk2slot = map_d.as<int2>() + bc.s + bc.u;
    A.tmaps = tmaps_d.as<CUtensorMap>();
    A.part = part_d.as<double>();
    A.ticket = ticket_d.as<unsigned>();
    A.n_active = counters_d.as<int>();
    A.part_stride = part_stride;
    return A;
  }

  int find_slots(int s) const {  // first fit of s contiguous free slots
    const int n = (int)owner.size();
    for (int a = 0; a + s <= n; ++a) {
      bool ok = true;
      for (int q = a; q < a + s && ok; ++q) ok = owner[q] < 0;
      if (ok) return a;
    }
    return -1;
  }

  size_t footprint(const Request& r) const {
    const int64_t nc = (int64_t)r.hx.size() * r.hy.size() * r.hz.size();
    const int64_t n1 = r.hx.size() + r.hy.size() + r.hz.size();
    size_t b = 9 * n1 * 12 + 7 * nc * 12 + nc * 8 + nc * 16;  // grid: geometry, masses, diag(K), sigma, packed masses
    b += 3 * nc * 8;                                         // f
    b += (size_t)r.s * slot_vector_bytes(nc, opt.solver.precision);
    b += 4096 + r.rx.size() * 16 * 8 + r.c.size() * 8 + (size_t)r.n_rx * r.K * 8;
    return b;
  }

  int admit(Request& r, int first) {
    cudaStream_t s_ = st;
    TEM_TRY(tem_build_grid(r.hx.data(), r.hx.size(), r.hy.data(), r.hy.size(), r.hz.data(), r.hz.size(), r.origin,
                           r.sigma.data(), s_, &r.grid));
    std::vector<Term> fterms;
    TEM_TRY(build_source(r.grid, r.loop.data(), (int64_t)r.loop.size() / 2, r.z_loop, r.current, fterms));
    std::vector<int64_t> tedge;
    std::vector<double> tw;
    std::vector<int> toff(1, 0);
    for (int q = 0; q < r.n_rx; ++q) {
      std::vector<Term> t;
      TEM_TRY(build_receiver(r.grid, r.rx.data() + 3 * q, t));
      for (auto& e : t) {
        tedge.push_back(e.edge);
        tw.push_back(e.w);
      }
      toff.push_back((int)tedge.size());
    }
    const int64_t nc = r.grid->v.ncomp;
    TEM_TRY(r.fbuf.alloc(3 * nc * sizeof(double), s_));
    const size_t per = slot_vector_bytes(nc, opt.solver.precision);
    TEM_TRY(r.vec.alloc(per * r.s, s_));
    const size_t nf = fterms.size(), nt = tedge.size();
    TEM_TRY(r.misc.alloc(256 + nf * 16 + nt * 16 + (r.n_rx + 1) * 8 + r.c.size() * 8 + (size_t)r.n_rx * r.K * 8 + 1024, s_));
    int64_t* d_fidx = r.misc.as<int64_t>();
    double* d_fval = reinterpret_cast<double*>(d_fidx + nf);
    r.d_tedge = reinterpret_cast<int64_t*>(d_fval + nf);
    r.d_tw = reinterpret_cast<double*>(r.d_tedge + nt);
    r.d_c = r.d_tw + nt;
    r.d_out = r.d_c + r.c.size();
    r.d_toff = reinterpret_cast<int*>(r.d_out + (size_t)r.n_rx * r.K);
    std::vector<int64_t> fi;
    std::vector<double> fv;
    double ff = 0;
    for (auto& t : fterms) {
      fi.push_back(t.edge);
      fv.push_back(t.w);
      ff += t.w * t.w;
    }
    TEM_CUDA_TRY(cudaMemsetAsync(r.fbuf.ptr, 0, 3 * nc * sizeof(double), s_));
    TEM_CUDA_TRY(cudaMemcpyAsync(d_fidx, fi.data(), nf * 8, cudaMemcpyHostToDevice, s_));
    TEM_CUDA_TRY(cudaMemcpyAsync(d_fval, fv.data(), nf * 8, cudaMemcpyHostToDevice, s_));
    if (nt) {
      TEM_CUDA_TRY(cudaMemcpyAsync(r.d_tedge, tedge.data(), nt * 8, cudaMemcpyHostToDevice, s_));
      TEM_CUDA_TRY(cudaMemcpyAsync(r.d_tw, tw.data(), nt * 8, cudaMemcpyHostToDevice, s_));
    }
    TEM_CUDA_TRY(cudaMemcpyAsync(r.d_toff, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice, s_));
    TEM_CUDA_TRY(cudaMemcpyAsync(r.d_c, r.c.data(), r.c.size() * 8, cudaMemcpyHostToDevice, s_));
    k_scatter<<<(int)((nf + 255) / 256 + 1), 256, 0, s_>>>(d_fidx, d_fval, (int64_t)nf, r.fbuf.as<double>());
    count_launch();
    TEM_CUDA_TRY(cudaGetLastError());
    TEM_CUDA_TRY(cudaMemsetAsync(r.vec.ptr, 0, per * r.s, s_));
    // slots
    for (int i = 0; i < r.s; ++i) {
      const int q = first + i;
      SlotDesc d;
      std::memset(&d, 0, sizeof(d));
      const SlotVectors v = carve_slot(r.vec.as<char>() + per * i, nc, opt.solver.precision);
      d.g = r.grid->v;
      d.xi_re = r.xi[2 * i];
      d.xi_im = r.xi[2 * i + 1];
      d.x = v.x; d.w = v.w; d.a0 = v.a0; d.a1 = v.a1; d.q = v.q;
      d.xn = v.xn; d.psi = v.psi; d.b0 = v.b0; d.b1 = v.b1; d.cn = v.cn; d.u = v.u; d.gp = v.gp;
      d.x64[0] = v.x64[0];
      d.x64[1] = v.x64[1];
      d.f = r.fbuf.as<double>();
      d.rhs_c = nullptr;
      d.nodal = nodal;
      d.fp64_inner = opt.solver.precision == TEM_PREC_FP64 ? 1 : 0;
      d.div_nx = make_fastdiv((uint32_t)d.g.nx);
      d.div_ny = make_fastdiv((uint32_t)d.g.ny);
      d.div_nynz = make_fastdiv((uint32_t)(d.g.ny * d.g.nz));
      decompose_slot(d, nodal);
      d.tma = 0;
      if (opt.solver.precision == TEM_PREC_MIXED && tma_stencil_enabled()) {
        CUtensorMap tm[tma::NMAP];
        if (encode_tile_maps(d, tm)) {
          d.tma = 1;
          TEM_CUDA_TRY(cudaMemcpyAsync(tmaps_d.as<CUtensorMap>() + (size_t)q * tma::NMAP, tm, sizeof(tm),
                                       cudaMemcpyHostToDevice, s_));
          TEM_CUDA_TRY(cudaStreamSynchronize(s_));   // tm lives on this stack frame
        }
      }
      SlotScalars S;
      std::memset(&S, 0, sizeof(S));
      S.max_iter = opt.solver.max_iter;
      S.ff = ff;
      S.tol_outer2 = opt.solver.tol * opt.solver.tol * ff;
      S.inner_rel2 = opt.solver.inner_tol * opt.solver.inner_tol;
      S.scale = 1.0 / std::sqrt(ff);
      S.inv_scale_prev = 1.0;
      S.max_outer = opt.solver.max_outer;
      S.stall_window = TEM_STALL_WINDOW;
      S.carry = opt.solver.carry_direction != 0;
      S.stalled = 0;
      S.carry_ratio = 0.0;
      slots_h[q] = d;
      sc_h[q] = S;
      owner[q] = (int)r.ticket;
      TEM_CUDA_TRY(cudaMemcpyAsync(sc_d.as<SlotScalars>() + q, &sc_h[q], sizeof(SlotScalars), cudaMemcpyHostToDevice, s_));
    }
    r.first_slot = first;
    maps_dirty = true;
    return TEM_OK;
  }

  // The slots to launch: those of running requests whose shifts have not finished.
  std::vector<char> wanted_slots() const {
    std::vector<char> use(owner.size(), 0);
    for (size_t q = 0; q < owner.size(); ++q) use[q] = owner[q] >= 0 && !sc_h[q].done;
    return use;
  }

  int rebuild_maps() {
    // interleaved block lists of the wanted slots; slot descriptors of the table
    in_maps = wanted_slots();
    std::vector<int2> map;
    build_block_maps(slots_h, in_maps, map, &bc);
    if (map.empty()) map.push_back(make_int2(0, 0));
    if (map_d.bytes < map.size() * sizeof(int2)) TEM_TRY(map_d.alloc(2 * map.size() * sizeof(int2), st));
    TEM_CUDA_TRY(cudaMemcpyAsync(map_d.ptr, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    TEM_CUDA_TRY(cudaMemcpyAsync(slots_d.ptr, slots_h.data(), slots_h.size() * sizeof(SlotDesc),
                                 cudaMemcpyHostToDevice, st));
    TEM_CUDA_TRY(cudaStreamSynchronize(st));   // map lives on this stack frame
    maps_dirty = false;
    return TEM_OK;
  }

  int launch_residual_and_start() {
    BatchArgs A = args();
    int* n_done = counters_d.as<int>() + 1;
    if (bc.s == 0) return TEM_OK;
    if (opt.solver.precision == TEM_PREC_FP64) {
      k_residual<double><<<bc.s, NT, 0, st>>>(A, n_done);
      if (nodal) k_cocg_nodal<double, true><<<bc.n, NT, 0, st>>>(A);
    } else {
      k_residual<float><<<bc.s, NT, 0, st>>>(A, n_done);
      if (nodal) k_cocg_nodal<float, true><<<bc.n, NT, 0, st>>>(A);
    }
    count_launch(nodal ? 2 : 1);
    TEM_CUDA_TRY(cudaGetLastError());
    return TEM_OK;
  }

  int launch_iteration() {
    BatchArgs A = args();
    if (bc.s == 0) return TEM_OK;
    if (opt.solver.precision == TEM_PREC_FP64) {
      k_cocg_stencil<double><<<bc.s, NT, 0, st>>>(A);
      k_cocg_update<double><<<bc.u, NT, 0, st>>>(A);
      count_launch(2);
      TEM_CUDA_TRY(cudaGetLastError());
      return TEM_OK;
    }
    TEM_TRY(launch_pass_a_f32(A, bc, nodal != 0, st));
    return launch_pass_b_f32(A, bc, st);
  }

  int finish(Request& r) {
    k_project_combine<<<r.n_rx, 128, 0, st>>>(slots_d.as<SlotDesc>() + r.first_slot,
                                               sc_d.as<SlotScalars>() + r.first_slot, r.s, r.d_tedge, r.d_tw,
                                               r.d_toff, r.d_c, r.K, r.d_out, r.n_rx);
    count_launch();
    TEM_CUDA_TRY(cudaGetLastError());
    r.d.assign((size_t)r.n_rx * r.K, 0.0);
    TEM_CUDA_TRY(cudaMemcpyAsync(r.d.data(), r.d_out, r.d.size() * 8, cudaMemcpyDeviceToHost, st));
    TEM_CUDA_TRY(cudaStreamSynchronize(st));
    r.status = TEM_OK;
    for (int i = 0; i < r.s; ++i) {
      const SlotScalars& S = sc_h[r.first_slot + i];
      r.max_iters = std::max(r.max_iters, (int)S.total_iters);
      if (S.status == TEM_ETIMEOUT) r.status = TEM_ETIMEOUT;
      else if (S.status == TEM_EBREAKDOWN && r.status != TEM_ETIMEOUT) r.status = TEM_EBREAKDOWN;
      else if (S.status == TEM_ENOCONV && r.status == TEM_OK) r.status = TEM_ENOCONV;
      owner[r.first_slot + i] = -1;
    }
    r.t_done = now_s();
    r.fbuf.release();
    r.vec.release();
    r.misc.release();
    if (r.grid) {
      tem_grid_destroy(r.grid);
      r.grid = nullptr;
    }
    used -= r.footprint;
    maps_dirty = true;
    return TEM_OK;
  }

  int step() {
    // admit in arrival order while slots and memory allow
    while (!queue.empty()) {
      Request& r = *queue.front();
      const int first = find_slots(r.s);
      if (first < 0 || used + r.footprint > (size_t)opt.hbm_budget_bytes) {
        if (running.empty() && (first < 0 || r.footprint > (size_t)opt.hbm_budget_bytes)) {
          // can never fit: fail it instead of waiting forever
          r.status = TEM_ENOMEM;
          r.t_admit = r.t_done = now_s();
          finished[r.ticket] = std::move(queue.front());
          queue.pop_front();
          continue;
        }
        break;
      }
      r.t_admit = now_s();
      const int rc = admit(r, first);
      if (rc != TEM_OK) {
        for (int i = 0; i < r.s; ++i)
          if (owner[first + i] == (int)r.ticket) owner[first + i] = -1;
        r.status = rc;
        r.t_done = now_s();
        finished[r.ticket] = std::move(queue.front());
        queue.pop_front();
        continue;
      }
      used += r.footprint;
      running.push_back(std::move(queue.front()));
      queue.pop_front();
    }
    if (running.empty()) return TEM_OK;
    if (maps_dirty || wanted_slots() != in_maps) TEM_TRY(rebuild_maps());
    TEM_TRY(launch_residual_and_start());
    for (int it = 0; it < opt.iters_per_step; ++it) TEM_TRY(launch_iteration());
    TEM_TRY(launch_residual_and_start());
    TEM_CUDA_TRY(cudaMemcpyAsync(sc_h.data(), sc_d.ptr, sc_h.size() * sizeof(SlotScalars), cudaMemcpyDeviceToHost, st));
    TEM_CUDA_TRY(cudaStreamSynchronize(st));
    // finish requests whose shifts are all done
    for (size_t q = 0; q < running.size();) {
      Request& r = *running[q];
      bool all = true;
      for (int i = 0; i < r.s && all; ++i) all = sc_h[r.first_slot + i].done != 0;
      if (!all) {
        ++q;
        continue;
      }
      TEM_TRY(finish(r));
      finished[r.ticket] = std::move(running[q]);
      running.erase(running.begin() + q);
    }
    return TEM_OK;
  }
};

extern "C" {

void tem_server_default_options(tem_server_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = 0;
  }
  opt->hbm_budget_bytes = (int64_t)(0.8 * (double)fr);
  opt->max_slots = 128;
  opt->iters_per_step = 32;
  tem_default_options(&opt->solver);
  opt->solver.precision = TEM_PREC_MIXED;
}

int tem_server_create(const tem_server_options* opt_in, void* cuda_stream, tem_server** out) {
  if (!out) return TEM_EINVAL;
  *out = nullptr;
  tem_server_options opt;
  tem_server_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.max_slots < 1 || opt.max_slots > 1024 || opt.iters_per_step < 1 || opt.hbm_budget_bytes <= 0)
    return TEM_EINVAL;
  if (opt.solver.precision != TEM_PREC_FP64 && opt.solver.precision != TEM_PREC_MIXED) return TEM_EINVAL;
  if (!(opt.solver.tol > 0 && opt.solver.tol < 1) || !(opt.solver.inner_tol > 0 && opt.solver.inner_tol < 1))
    return TEM_EINVAL;
  std::unique_ptr<tem_server> s(new tem_server());
  s->opt = opt;
  s->st = static_cast<cudaStream_t>(cuda_stream);
  s->nodal = opt.solver.precond == TEM_PRECOND_JACOBI ? 0 : 1;
  const int n = opt.max_slots;
  s->slots_h.assign(n, SlotDesc());
  std::memset(s->slots_h.data(), 0, n * sizeof(SlotDesc));
  s->sc_h.assign(n, SlotScalars());
  std::memset(s->sc_h.data(), 0, n * sizeof(SlotScalars));
  for (auto& S : s->sc_h) S.done = 1;  // free slots never run
  s->owner.assign(n, -1);
  TEM_TRY(s->slots_d.alloc(n * sizeof(SlotDesc), s->st));
  TEM_TRY(s->sc_d.alloc(n * sizeof(SlotScalars), s->st));
  TEM_TRY(s->part_d.alloc((size_t)n * s->part_stride * sizeof(double), s->st));
  TEM_TRY(s->ticket_d.alloc(n * sizeof(unsigned), s->st));
  TEM_TRY(s->counters_d.alloc(2 * sizeof(int), s->st));
  TEM_TRY(s->tmaps_d.alloc((size_t)n * tma::NMAP * sizeof(CUtensorMap), s->st));
  TEM_CUDA_TRY(cudaMemcpyAsync(s->sc_d.ptr, s->sc_h.data(), n * sizeof(SlotScalars), cudaMemcpyHostToDevice, s->st));
  TEM_CUDA_TRY(cudaMemsetAsync(s->ticket_d.ptr, 0, n * sizeof(unsigned), s->st));
  TEM_CUDA_TRY(cudaMemsetAsync(s->counters_d.ptr, 0, 2 * sizeof(int), s->st));
  TEM_CUDA_TRY(cudaStreamSynchronize(s->st));
  *out = s.release();
  return TEM_OK;
}

int tem_server_submit(tem_server* srv, const double* hx, int64_t nx, const double* hy, int64_t ny, const double* hz,
                      int64_t nz, const double* origin, const double* sigma, const double* loop_xy,
                      int64_t n_vertices, double z_loop, double current, const double* rx_xyz, int64_t n_rx,
                      const double* xi, const double* c, int64_t s, int64_t K, int64_t* ticket_out) {
  if (!srv || !hx || !hy || !hz || !origin || !sigma || !loop_xy || !rx_xyz || !xi || !c || !ticket_out)
    return TEM_EINVAL;
  if (nx < 2 || ny < 2 || nz < 2 || nx > 4096 || ny > 4096 || nz > 4096) return TEM_EINVAL;
  if (3 * nx * ny * nz >= (int64_t(1) << 31)) return TEM_EINVAL;
  if (s < 1 || s > 64 || s > srv->opt.max_slots || K < 1 || K > 100000 || n_rx < 1 || n_rx > 4096) return TEM_EINVAL;
  if (!all_finite_positive(hx, nx) || !all_finite_positive(hy, ny) || !all_finite_positive(hz, nz) ||
      !all_finite_positive(sigma, nx * ny * nz))
    return TEM_EINVAL;
  for (int64_t q = 0; q < 2 * s; ++q)
    if (!std::isfinite(xi[q])) return TEM_EINVAL;
  for (int64_t q = 0; q < s; ++q)
    if (xi[2 * q] >= 0.0 && xi[2 * q + 1] == 0.0) return TEM_EINVAL;
  for (int64_t q = 0; q < 2 * s * K; ++q)
    if (!std::isfinite(c[q])) return TEM_EINVAL;
  std::unique_ptr<Request> r(new Request());
  r->hx.assign(hx, hx + nx);
  r->hy.assign(hy, hy + ny);
  r->hz.assign(hz, hz + nz);
  for (int q = 0; q < 3; ++q) r->origin[q] = origin[q];
  r->sigma.assign(sigma, sigma + nx * ny * nz);
  r->loop.assign(loop_xy, loop_xy + 2 * n_vertices);
  r->rx.assign(rx_xyz, rx_xyz + 3 * n_rx);
  r->xi.assign(xi, xi + 2 * s);
  r->c.assign(c, c + 2 * s * K);
  r->z_loop = z_loop;
  r->current = current;
  r->s = (int)s;
  r->K = (int)K;
  r->n_rx = (int)n_rx;
  {  // geometry checks on the host, before anything reaches the device
    HostGrid hg(*r);
    SlotDesc probe;
    std::memset(&probe, 0, sizeof(probe));
    probe.g = hg.g.v;
    decompose_slot(probe, srv->nodal);
    if (probe.nblk_stencil > kMaxBlocksPerSlot || probe.nblk_update > kMaxBlocksPerSlot ||
        probe.nblk_nodal > kMaxBlocksPerSlot)
      return TEM_EINVAL;  // larger than one server slot's reduction buffers
    std::vector<Term> t;
    TEM_TRY(build_source(&hg.g, loop_xy, n_vertices, z_loop, current, t));
    for (int64_t q = 0; q < n_rx; ++q) TEM_TRY(build_receiver(&hg.g, rx_xyz + 3 * q, t));
  }
  r->footprint = srv->footprint(*r);
  r->ticket = srv->next_ticket++;
  r->t_submit = now_s();
  *ticket_out = r->ticket;
  srv->queue.push_back(std::move(r));
  return TEM_OK;
}

int tem_server_step(tem_server* srv) {
  if (!srv) return TEM_EINVAL;
  return srv->step();
}

int tem_server_poll(tem_server* srv, int64_t ticket, double* dbzdt_out, tem_request_stats* stats) {
  if (!srv) return TEM_EINVAL;
  auto it = srv->finished.find(ticket);
  if (it == srv->finished.end()) {
    for (auto& r : srv->queue)
      if (r->ticket == ticket) return TEM_EBUSY;
    for (auto& r : srv->running)
      if (r->ticket == ticket) return TEM_EBUSY;
    return TEM_EINVAL;
  }
  Request& r = *it->second;
  if (dbzdt_out && !r.d.empty()) std::memcpy(dbzdt_out, r.d.data(), r.d.size() * sizeof(double));
  if (stats) {
    stats->submit_s = r.t_submit;
    stats->admit_s = r.t_admit;
    stats->done_s = r.t_done;
    stats->footprint_bytes = (int64_t)r.footprint;
    stats->status = r.status;
    stats->max_iters = r.max_iters;
  }
  const int st = r.status;
  srv->finished.erase(it);
  return st;
}

int tem_server_counts(const tem_server* srv, int64_t* queued, int64_t* running, int64_t* done) {
  if (!srv) return TEM_EINVAL;
  if (queued) *queued = (int64_t)srv->queue.size();
  if (running) *running = (int64_t)srv->running.size();
  if (done) *done = (int64_t)srv->finished.size();
  return TEM_OK;
}

int tem_server_destroy(tem_server* srv) {
  if (!srv) return TEM_EINVAL;
  cudaStreamSynchronize(srv->st);
  delete srv;
  return TEM_OK;
}

}  // extern "C"
