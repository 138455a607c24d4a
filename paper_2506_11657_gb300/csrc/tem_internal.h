// Internal structures of the TEM library (device layout, solver state, helpers).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include <string>

#include "../../include/tem.h"

#define TEM_MU0 (4e-7 * 3.14159265358979323846)

namespace tem {

// ---- error plumbing ------------------------------------------------------
struct Status {
  int code = TEM_OK;
};

#define TEM_CUDA_TRY(expr)                                       \
  do {                                                           \
    cudaError_t err__ = (expr);                                  \
    if (err__ != cudaSuccess) {                                  \
      tem::set_last_error(cudaGetErrorString(err__), __FILE__, __LINE__); \
      return TEM_ECUDA;                                          \
    }                                                            \
  } while (0)

#define TEM_TRY(expr)               \
  do {                              \
    int st__ = (expr);              \
    if (st__ != TEM_OK) return st__; \
  } while (0)

void set_last_error(const char* msg, const char* file, int line);

// A named NVTX range for the lifetime of the object (visible in Nsight timelines; no cost
// without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- device memory ---------------------------------------------------------
void* dev_alloc(size_t bytes, cudaStream_t stream);
void dev_free(void* p, size_t bytes, cudaStream_t stream);

// A device buffer owned by the library (freed on the stream it was made on).
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  int alloc(size_t nbytes, cudaStream_t s);
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// ---- grid ------------------------------------------------------------------
// Plain-old-data view of a grid, passed by value to kernels.
struct GridView {
  int nx, ny, nz;
  int64_t ncomp;            // nx*ny*nz entries per edge direction
  // 1-D geometry (device): edge lengths and dual lengths at node planes 0..n-1
  const double* Lx; const double* Ly; const double* Lz;
  const double* Sx; const double* Sy; const double* Sz;
  const float* Lxf; const float* Lyf; const float* Lzf;
  const float* Sxf; const float* Syf; const float* Szf;
  const double* Rx; const double* Ry; const double* Rz;   // 1 / L
  const float* Rxf; const float* Ryf; const float* Rzf;
  const double* Me;         // [3][ncomp] lumped edge mass, 0 on boundary/padding entries
  const float* Mef;         // FP32 copy
  const double* Wn;         // [ncomp] per node: sum over its edges of M_e / L_e^2 (0 on boundary nodes)
  const float* Wnf;         // FP32 copy
  const double* dK;         // [3][ncomp] diag(K) per edge, 0 on boundary/padding entries
  const float* dKf;         // FP32 copy
  const float4* Mq;         // [ncomp] per node (M_x, M_y, M_z, W_n) in FP32: the masses of the three
                            // edges leaving the node and its nodal weight, one 16-byte record
};

}  // namespace tem

struct tem_grid {
  tem::GridView v;
  std::vector<double> hx, hy, hz;   // host copies
  double origin[3];
  std::vector<double> sigma;        // host copy (for the adjoint)
  tem::DevBuf geo;                  // packed 1-D arrays
  tem::DevBuf me;                   // Me, Wn, dK (FP64) then Mef, Wnf, dKf (FP32)
  tem::DevBuf sig;                  // sigma on the device (FP64)
  tem::DevBuf mq;                   // packed FP32 (M_x, M_y, M_z, W_n) per node
  uint64_t sigma_gen = 0;           // incremented by every conductivity upload
  int device = 0;
};

namespace tem {

// Complex helpers usable on host and device.
template <class T> struct cplx { T re, im; };

// Host-side geometry helpers (grid.cu)
int locate_node(const std::vector<double>& h, double origin, double v, int* idx);
// Sparse term lists in the device edge layout (unique edges, boundary edges dropped).
struct Term { int64_t edge; double w; };
int build_source(const tem_grid* g, const double* loop_xy, int64_t nv, double z_loop, double current,
                 std::vector<Term>& f);
int build_receiver(const tem_grid* g, const double* xyz, std::vector<Term>& q);

// Unsigned 32-bit division by a run-time constant through a precomputed
// multiplier (Granlund & Montgomery 1994): q = (umulhi(n, m) + n) >> s.
struct FastDiv {
  uint32_t d, m, s;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  f.s = s;
  f.m = (uint32_t)((((1ull << s) - d) << 32) / d + 1);
  return f;
}
__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(n, f.m);
#else
  const uint32_t t = (uint32_t)(((uint64_t)n * f.m) >> 32);
#endif
  return (uint32_t)(((uint64_t)t + n) >> f.s);
}

// ---- batched COCG ----------------------------------------------------------
// One "slot" = one shifted system (a problem and a shift).  All slots of a
// batch advance together: one stencil pass and one update pass per iteration.
struct SlotDesc {
  GridView g;
  double xi_re, xi_im;      // shift
  // inner COCG vectors (precision T): edge part and nodal part of the iterate and directions
  void* x;                  // edge part of the correction
  void* w;                  // D^{-1} r, the Jacobi-scaled residual (r = D w is rebuilt where needed)
  void* a0; void* a1;       // edge part of the search direction, double-buffered
  void* q;                  // A p
  void* xn;                 // nodal part of the correction (x = x_e + G x_n)
  void* psi;                // D_n^{-1} G^T r
  void* b0; void* b1;       // nodal part of the search direction, double-buffered
  void* cn;                 // G^T of the inner right-hand side, s xi G^T M x64 (set when a solve starts)
  void* u;                  // v = cn + xi G^T M d: the start pass sets it to cn, the update pass adds
                            // alpha xi G^T M p with the correction (so G^T r = v)
  void* gp;                 // G^T M p of the current direction, from the stencil pass
  int tiles_x, tiles_y, zchunks;  // stencil decomposition
  int zchunk;               // planes per stencil CTA (a function of this slot's grid only)
  int nblk_stencil;         // tiles_x*tiles_y*zchunks
  int nblk_update;          // blocks of the update pass
  int nblk_nodal;           // blocks of the nodal pass
  int tma;                  // 1: the FP32 stencil pass may use this slot's tile maps (even nx)
  FastDiv div_nx, div_ny, div_nynz;
  // defect correction (FP64 outer loop)
  const double* f;          // right-hand side, real, edge layout (FP64)
  const double* rhs_c;      // complex right-hand side (adjoint, linearised forward), or NULL
  int rhs_div;              // 1: the right-hand side may have G^T b != 0 (linearised forward)
  void* x64[2];             // FP64 iterate, double-buffered by the residual pass
  int nodal;                // 1: preconditioner with the nodal-gradient correction; 0: Jacobi only
  int fp64_inner;           // 1: inner sweeps in FP64 (aim at the final tolerance directly)
};

struct SlotScalars {
  double rho_re, rho_im;    // (r, z) of the current iterate
  double alpha_re, alpha_im;
  double beta_re, beta_im;
  double rhoe_re, rhoe_im;  // edge part r^T D^{-1} r, from the update (or residual) pass
  double rr;                // ||r||^2 (recursive)
  double bb;                // ||b||^2 of this solve's right-hand side
  double tol2;              // stop when rr <= tol2
  int32_t active;           // 1 while iterating
  int32_t pending;          // 1 after the residual pass armed an inner solve that the nodal pass has not started
  int32_t iters;
  int32_t max_iter;
  int32_t status;           // TEM_OK / TEM_ENOCONV / TEM_EBREAKDOWN
  int32_t parity;           // which direction buffer holds the current direction
  int32_t xcur;             // which x64 buffer holds the current FP64 iterate
  // outer (FP64 residual) loop
  double ff;                // ||f||^2
  double tol_outer2;        // stop when ||f - A x||^2 <= tol_outer2 (= tol^2 ||f||^2)
  double inner_rel2;        // inner solves stop at ||r_inner||^2 <= inner_rel2 * ||r_start||^2
  double rr64;              // last FP64 residual norm^2
  double scale;             // inner right-hand side = scale * r64
  double inv_scale_prev;    // correction of the last inner solve = inv_scale_prev * delta
  int32_t outer;            // outer steps taken
  int32_t max_outer;
  int32_t done;             // 1 once the FP64 residual met the tolerance (or the slot failed)
  int32_t total_iters;      // inner iterations summed over outer steps
  double rr_best;           // smallest recursive ||r||^2 of the current inner solve
  int32_t it_best;          // iteration that reached it
  int32_t stall_window;     // end the inner solve after this many iterations without a new best
  int32_t carry;            // keep the search direction across outer steps (residual replacement)
  int32_t stalled;          // the last inner solve ended on stagnation
  double carry_ratio;       // s_prev / s of an armed solve that continues the direction, else 0
  // The update pass adds alpha p to the correction d on odd iterations only, two directions at
  // a time (both are still in the direction buffers), so an inner solve that ends after an even
  // iteration leaves its last term to the residual pass.
  double alpha_prev_re, alpha_prev_im;   // alpha of the last completed iteration
  int32_t lag;              // 1: d lacks alpha_prev p of the last completed iteration
  int32_t lag_par;          // parity of that iteration (its direction is in a0/b0 if 1, else a1/b1)
};

}  // namespace tem
