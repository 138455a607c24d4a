// Grid construction, allocator, status strings, and host-side geometry helpers.
//
// Sec. 2.2: the lumped mass M_e = sum_{cells c containing e} sigma_c V_c / 4 and
// the 1-D factors of K (edge lengths L and dual lengths L*) of the Yee grid.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <algorithm>

#include "tem_internal.h"
#include "solver.h"

namespace tem {

// ---------------------------------------------------------------- errors
static thread_local char g_last_error[512] = {0};

void set_last_error(const char* msg, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s:%d)", msg, file, line);
}

// -------------------------------------------------------------- allocator
static tem_alloc_fn g_alloc = nullptr;
static tem_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::once_flag g_pool_once;

void* dev_alloc(size_t bytes, cudaStream_t stream) {
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc(bytes, stream, g_alloc_ctx);
  std::call_once(g_pool_once, [] {
    // keep freed blocks in the stream-ordered pool instead of returning them to the driver
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t stream) {
  if (!p) return;
  if (g_free) {
    g_free(p, bytes, stream, g_alloc_ctx);
    return;
  }
  cudaFreeAsync(p, stream);
}

int DevBuf::alloc(size_t nbytes, cudaStream_t s) {
  release();
  ptr = dev_alloc(nbytes, s);
  if (!ptr) return TEM_ENOMEM;
  bytes = nbytes;
  stream = s;
  return TEM_OK;
}

void DevBuf::release() {
  if (ptr) dev_free(ptr, bytes, stream);
  ptr = nullptr;
  bytes = 0;
}

// ----------------------------------------------------------- device mass
__global__ void k_mass(int nx, int ny, int nz, const double* hx, const double* hy, const double* hz,
                       const double* sigma, double* Me, float* Mef) {
  const int64_t ncomp = (int64_t)nx * ny * nz;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * ncomp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = int(e / ncomp);
    const int64_t r = e - c * ncomp;
    const int i = int(r % nx);
    const int64_t r2 = r / nx;
    const int j = int(r2 % ny), k = int(r2 / ny);
    double m = 0.0;
    bool valid = c == 0 ? (j > 0 && k > 0) : (c == 1 ? (i > 0 && k > 0) : (i > 0 && j > 0));
    if (valid) {
      // the four cells around the edge: offsets in the two transverse directions
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          int ci = i, cj = j, ck = k;
          if (c == 0) { cj = j - 1 + a; ck = k - 1 + b; }
          if (c == 1) { ci = i - 1 + a; ck = k - 1 + b; }
          if (c == 2) { ci = i - 1 + a; cj = j - 1 + b; }
          const int64_t cell = ci + (int64_t)nx * (cj + (int64_t)ny * ck);
          m += 0.25 * sigma[cell] * hx[ci] * hy[cj] * hz[ck];
        }
    }
    Me[e] = m;
    Mef[e] = float(m);
  }
}

// W_n = sum over the six edges at node n of M_e / L_e^2 (interior nodes; 0 on the boundary):
// the diagonal of G^T M G for the nodal gradient G.
__global__ void k_node_weight(int nx, int ny, int nz, const double* hx, const double* hy, const double* hz,
                              const double* Me, double* Wn, float* Wnf) {
  const int64_t ncomp = (int64_t)nx * ny * nz;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ncomp; n += (int64_t)gridDim.x * blockDim.x) {
    const int i = int(n % nx);
    const int64_t r = n / nx;
    const int j = int(r % ny), k = int(r / ny);
    double w = 0.0;
    if (i > 0 && j > 0 && k > 0) {
      w = Me[n - 1] / (hx[i - 1] * hx[i - 1]) + Me[n] / (hx[i] * hx[i]) +
          Me[ncomp + n - nx] / (hy[j - 1] * hy[j - 1]) + Me[ncomp + n] / (hy[j] * hy[j]) +
          Me[2 * ncomp + n - (int64_t)nx * ny] / (hz[k - 1] * hz[k - 1]) + Me[2 * ncomp + n] / (hz[k] * hz[k]);
    }
    Wn[n] = w;
    Wnf[n] = float(w);
  }
}

// diag(K) per edge (Sec. 2.2: K = C^T diag(L*/(mu0 A)) C, so K_ee = L_e^2 sum_{f ni e} L*_f/(mu0 A_f));
// 0 on boundary and padding entries.
__global__ void k_diagK(int nx, int ny, int nz, const double* L, const double* S, double* dK, float* dKf) {
  const int64_t ncomp = (int64_t)nx * ny * nz;
  const double* Lx = L; const double* Ly = L + nx; const double* Lz = L + nx + ny;
  const double* Sx = S; const double* Sy = S + nx; const double* Sz = S + nx + ny;
  const double im = 1.0 / TEM_MU0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * ncomp; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = int(e / ncomp);
    const int64_t r = e - c * ncomp;
    const int i = int(r % nx);
    const int64_t r2 = r / nx;
    const int j = int(r2 % ny), k = int(r2 / ny);
    double v = 0.0;
    if (c == 0 && j > 0 && k > 0)
      v = Lx[i] * im * (Sz[k] * (1.0 / Ly[j] + 1.0 / Ly[j - 1]) + Sy[j] * (1.0 / Lz[k] + 1.0 / Lz[k - 1]));
    if (c == 1 && i > 0 && k > 0)
      v = Ly[j] * im * (Sz[k] * (1.0 / Lx[i] + 1.0 / Lx[i - 1]) + Sx[i] * (1.0 / Lz[k] + 1.0 / Lz[k - 1]));
    if (c == 2 && i > 0 && j > 0)
      v = Lz[k] * im * (Sx[i] * (1.0 / Ly[j] + 1.0 / Ly[j - 1]) + Sy[j] * (1.0 / Lx[i] + 1.0 / Lx[i - 1]));
    dK[e] = v;
    dKf[e] = float(v);
  }
}

// (M_x, M_y, M_z, W_n) per node in one FP32 record: the tile loads of the FP32 stencil pass
// fetch the masses a node's edges need as one 16-byte element.
__global__ void k_pack_mass(int64_t ncomp, const float* Mef, const float* Wnf, float4* Mq) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < ncomp; n += (int64_t)gridDim.x * blockDim.x)
    Mq[n] = make_float4(Mef[n], Mef[ncomp + n], Mef[2 * ncomp + n], Wnf[n]);
}

static bool finite_positive(const double* a, int64_t n) {
  for (int64_t q = 0; q < n; ++q)
    if (!(std::isfinite(a[q]) && a[q] > 0.0)) return false;
  return true;
}

int locate_node(const std::vector<double>& h, double origin, double v, int* idx) {
  // nearest node coordinate; EINVAL unless within 1e-9 of the extent
  double x = origin, best = std::fabs(v - origin);
  int bi = 0;
  for (size_t q = 0; q < h.size(); ++q) {
    x += h[q];
    const double dd = std::fabs(v - x);
    if (dd < best) { best = dd; bi = int(q) + 1; }
  }
  double ext = 0.0;
  for (double w : h) ext += w;
  if (best > 1e-9 * ext) return TEM_EINVAL;
  *idx = bi;
  return TEM_OK;
}

}  // namespace tem

using namespace tem;

static int upload_sigma(tem_grid* g, const double* sigma, cudaStream_t st) {
  const int64_t ncell = g->v.ncomp;
  if (!sigma || !finite_positive(sigma, ncell)) return TEM_EINVAL;
  g->sigma.assign(sigma, sigma + ncell);
  g->sigma_gen += 1;
  TEM_CUDA_TRY(cudaMemcpyAsync(g->sig.ptr, sigma, ncell * sizeof(double), cudaMemcpyHostToDevice, st));
  // layout: Me (3n), Wn (n), dK (3n) doubles, then Mef (3n), Wnf (n), dKf (3n) floats
  double* Me = g->me.as<double>();
  double* Wn = Me + 3 * ncell;
  float* Mef = reinterpret_cast<float*>(Wn + 4 * ncell);
  float* Wnf = Mef + 3 * ncell;
  const double* geo = g->geo.as<double>();
  const int nx = g->v.nx, ny = g->v.ny, nz = g->v.nz;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((3 * ncell + threads - 1) / threads, 152 * 32);
  k_mass<<<(int)blocks, threads, 0, st>>>(nx, ny, nz, geo, geo + nx, geo + nx + ny, g->sig.as<double>(), Me, Mef);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  k_node_weight<<<(int)std::min<int64_t>((ncell + threads - 1) / threads, 152 * 32), threads, 0, st>>>(
      nx, ny, nz, geo, geo + nx, geo + nx + ny, Me, Wn, Wnf);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  k_pack_mass<<<(int)std::min<int64_t>((ncell + threads - 1) / threads, 152 * 32), threads, 0, st>>>(
      ncell, Mef, Wnf, g->mq.as<float4>());
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}

extern "C" {

const char* tem_status_string(int status) {
  switch (status) {
    case TEM_OK: return "TEM_OK";
    case TEM_EINVAL: return "TEM_EINVAL: invalid argument";
    case TEM_ENOMEM: return "TEM_ENOMEM: device allocation failed";
    case TEM_ENOCONV: return "TEM_ENOCONV: a shifted solve reached max_iter";
    case TEM_EBREAKDOWN: return "TEM_EBREAKDOWN: COCG breakdown";
    case TEM_ETIMEOUT: return "TEM_ETIMEOUT: a bounded wait ran out";
    case TEM_ECUDA: return "TEM_ECUDA: CUDA runtime error";
    case TEM_EBUSY: return "TEM_EBUSY: not finished";
    default: return "unknown status";
  }
}

const char* tem_last_error(void) { return g_last_error; }

const char* tem_version(void) { return "tem-gb300 0.1 (sm_103a)"; }

int tem_set_allocator(tem_alloc_fn alloc, tem_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return TEM_EINVAL;
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return TEM_OK;
}

void tem_default_options(tem_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = TEM_PREC_FP64;
  opt->max_iter = 20000;
  opt->tol = 1e-12;
  opt->inner_tol = 1e-1;
  opt->max_outer = 40;
  opt->check_every = 32;
  opt->keep_state = 0;
  opt->carry_direction = 1;
}

int tem_build_grid(const double* hx, int64_t nx, const double* hy, int64_t ny, const double* hz, int64_t nz,
                   const double* origin, const double* sigma, void* cuda_stream, tem_grid** out) {
  if (!out || !hx || !hy || !hz || !origin || !sigma) return TEM_EINVAL;
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2) return TEM_EINVAL;
  if (nx > 4096 || ny > 4096 || nz > 4096) return TEM_EINVAL;
  if (3 * nx * ny * nz >= (int64_t(1) << 31)) return TEM_EINVAL;  // 32-bit entry indexing in the update pass
  if (!finite_positive(hx, nx) || !finite_positive(hy, ny) || !finite_positive(hz, nz)) return TEM_EINVAL;
  for (int q = 0; q < 3; ++q)
    if (!std::isfinite(origin[q])) return TEM_EINVAL;
  const int64_t ncell = nx * ny * nz;
  if (!finite_positive(sigma, ncell)) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  tem_grid* g = new tem_grid();
  g->hx.assign(hx, hx + nx);
  g->hy.assign(hy, hy + ny);
  g->hz.assign(hz, hz + nz);
  for (int q = 0; q < 3; ++q) g->origin[q] = origin[q];
  cudaGetDevice(&g->device);
  // packed 1-D geometry: L (3), S (3), 1/L (3) in FP64, then in FP32
  const int64_t n1 = nx + ny + nz;
  std::vector<double> geo(9 * n1);
  std::vector<float> geof(9 * n1);
  auto put = [&](int64_t off, const std::vector<double>& h) {
    const int64_t n = (int64_t)h.size();
    for (int64_t q = 0; q < n; ++q) {
      geo[off + q] = h[q];
      const double prev = q > 0 ? h[q - 1] : 0.0;
      geo[3 * n1 + off + q] = 0.5 * (prev + h[q]);  // dual length at node plane q
      geo[6 * n1 + off + q] = 1.0 / h[q];
    }
  };
  put(0, g->hx);
  put(nx, g->hy);
  put(nx + ny, g->hz);
  for (int64_t q = 0; q < 9 * n1; ++q) geof[q] = float(geo[q]);
  int rc = g->geo.alloc(9 * n1 * (sizeof(double) + sizeof(float)), st);
  if (rc == TEM_OK) rc = g->me.alloc(7 * ncell * (sizeof(double) + sizeof(float)), st);
  if (rc == TEM_OK) rc = g->sig.alloc(ncell * sizeof(double), st);
  if (rc == TEM_OK) rc = g->mq.alloc(ncell * sizeof(float4), st);
  if (rc != TEM_OK) {
    delete g;
    return rc;
  }
  double* gd = g->geo.as<double>();
  float* gf = reinterpret_cast<float*>(gd + 9 * n1);
  if (cudaMemcpyAsync(gd, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(gf, geof.data(), geof.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_last_error("geometry upload failed", __FILE__, __LINE__);
    delete g;
    return TEM_ECUDA;
  }
  GridView& v = g->v;
  v.nx = int(nx);
  v.ny = int(ny);
  v.nz = int(nz);
  v.ncomp = ncell;
  v.Lx = gd; v.Ly = gd + nx; v.Lz = gd + nx + ny;
  v.Sx = gd + 3 * n1; v.Sy = gd + 3 * n1 + nx; v.Sz = gd + 3 * n1 + nx + ny;
  v.Lxf = gf; v.Lyf = gf + nx; v.Lzf = gf + nx + ny;
  v.Sxf = gf + 3 * n1; v.Syf = gf + 3 * n1 + nx; v.Szf = gf + 3 * n1 + nx + ny;
  v.Rx = gd + 6 * n1; v.Ry = gd + 6 * n1 + nx; v.Rz = gd + 6 * n1 + nx + ny;
  v.Rxf = gf + 6 * n1; v.Ryf = gf + 6 * n1 + nx; v.Rzf = gf + 6 * n1 + nx + ny;
  v.Me = g->me.as<double>();
  v.Wn = v.Me + 3 * ncell;
  v.dK = v.Wn + ncell;
  v.Mef = reinterpret_cast<const float*>(v.dK + 3 * ncell);
  v.Wnf = v.Mef + 3 * ncell;
  v.dKf = v.Wnf + ncell;
  v.Mq = g->mq.as<float4>();
  {
    double* dK = const_cast<double*>(v.dK);
    float* dKf = const_cast<float*>(v.dKf);
    k_diagK<<<(int)std::min<int64_t>((3 * ncell + 255) / 256, 152 * 32), 256, 0, st>>>(
        int(nx), int(ny), int(nz), gd, gd + 3 * n1, dK, dKf);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      delete g;
      return TEM_ECUDA;
    }
  }
  rc = upload_sigma(g, sigma, st);
  if (rc == TEM_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = TEM_ECUDA;
  if (rc != TEM_OK) {
    delete g;
    return rc;
  }
  *out = g;
  return TEM_OK;
}

int tem_grid_set_sigma(tem_grid* grid, const double* sigma, void* cuda_stream) {
  if (!grid) return TEM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TEM_TRY(upload_sigma(grid, sigma, st));
  TEM_CUDA_TRY(cudaStreamSynchronize(st));
  return TEM_OK;
}

int tem_grid_dims(const tem_grid* grid, int64_t* dims) {
  if (!grid || !dims) return TEM_EINVAL;
  dims[0] = grid->v.nx;
  dims[1] = grid->v.ny;
  dims[2] = grid->v.nz;
  return TEM_OK;
}

int tem_grid_destroy(tem_grid* grid) {
  if (!grid) return TEM_EINVAL;
  cudaStreamSynchronize(grid->geo.stream);
  delete grid;
  return TEM_OK;
}

}  // extern "C"

