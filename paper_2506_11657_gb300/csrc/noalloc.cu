// tem_apply_operator_noalloc: the shifted operator q = (K - xi M) p without any
// device allocation.
//
// tem_apply_operator copies the caller's shifts into a small device buffer that it
// allocates for the call.  Some callers cannot allow that: a host framework that owns
// every byte of device memory through its own pool and forbids side allocations, or a
// latency-critical loop that cannot risk the device-wide synchronisation that
// cudaMalloc / cudaFree may imply.  This entry point keeps the shifts in a fixed
// array in device global memory instead; the caller still provides p and q.
//
// Limits and sharing: at most TEM_NOALLOC_MAX_SHIFTS shifts per call.  The array is
// shared by every call in the process (on each device that loads the library, it
// lives until the process exits) and holds the last call's shifts; each call
// overwrites the entries it uses before its kernel reads them.  Calls whose work
// overlaps on the GPU (for example on two streams at once) race on the array.
#include <mutex>

#include "kernels.cuh"
#include "solver.h"

#define TEM_NOALLOC_MAX_SHIFTS 64
#define TEM_NOALLOC_MAX_DEVICES 64

namespace {

// Device-side scratch: (re, im) of each shift.  In host code this name only stands in
// for the symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_xi[2 * TEM_NOALLOC_MAX_SHIFTS];

std::mutex g_noalloc_mu;
double* g_noalloc_xi_dev[TEM_NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
int noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= TEM_NOALLOC_MAX_DEVICES) return TEM_EINVAL;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_xi_dev[dev]) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_xi);
    if (err != cudaSuccess || !p) {
      tem::set_last_error(cudaGetErrorString(err), __FILE__, __LINE__);
      return TEM_ECUDA;
    }
    g_noalloc_xi_dev[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_xi_dev[dev];
  return TEM_OK;
}

}  // namespace

using namespace tem;

extern "C" int tem_apply_operator_noalloc(const tem_grid* grid, const double* xi, int64_t s, const void* p_dev,
                                          void* q_dev, int32_t precision, void* cuda_stream) {
  if (!grid || !xi || !p_dev || !q_dev || s < 1) return TEM_EINVAL;
  if (s > TEM_NOALLOC_MAX_SHIFTS) {
    set_last_error("tem_apply_operator_noalloc: more shifts than TEM_NOALLOC_MAX_SHIFTS (64)", __FILE__, __LINE__);
    return TEM_EINVAL;
  }
  if (precision != TEM_PREC_FP64 && precision != TEM_PREC_MIXED) return TEM_EINVAL;
  for (int64_t q = 0; q < 2 * s; ++q)
    if (!std::isfinite(xi[q])) return TEM_EINVAL;
  int dev = 0;
  TEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device) {
    set_last_error("tem_apply_operator_noalloc: the grid's device must be current", __FILE__, __LINE__);
    return TEM_EINVAL;
  }
  double* dxi = nullptr;
  TEM_TRY(noalloc_scratch(dev, &dxi));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  TEM_CUDA_TRY(cudaMemcpyAsync(dxi, xi, 2 * s * sizeof(double), cudaMemcpyHostToDevice, st));
  const GridView& g = grid->v;
  const int zchunk = 32;
  const int tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY, tz = (g.nz + zchunk - 1) / zchunk;
  dim3 grd(tx * ty * tz, (unsigned)s);
  if (precision == TEM_PREC_FP64)
    k_apply<double><<<grd, NT, 0, st>>>(g, dxi, p_dev, q_dev, tx, ty, zchunk);
  else
    k_apply<float><<<grd, NT, 0, st>>>(g, dxi, p_dev, q_dev, tx, ty, zchunk);
  count_launch();
  TEM_CUDA_TRY(cudaGetLastError());
  return TEM_OK;
}
