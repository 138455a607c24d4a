// Device kernels of the batched shifted COCG on the Yee edge grid.
//
// Operator (Sec. 2.2, the Nedelec/Yee discretisation of Eq. (pde)):
//   (A_i p)_e = (K p)_e - xi_i M_e p_e,
//   (K p)_e   = L_e * sum_{faces f containing e} (+-) F_f,
//   F_f       = (L*_f / mu0) * circ_f(p) / A_f   (written below with 1/L factors),
// with circ_f the signed sum of L_e p_e around face f.  For the face whose
// normal is +x at node (i, j, k):
//   F_x = (Sx_i/mu0) [ (p_y(i,j,k) - p_y(i,j,k+1)) / Lz_k + (p_z(i,j+1,k) - p_z(i,j,k)) / Ly_j ]
//   F_y = (Sy_j/mu0) [ (p_z(i,j,k) - p_z(i+1,j,k)) / Lx_i + (p_x(i,j,k+1) - p_x(i,j,k)) / Lz_k ]
//   F_z = (Sz_k/mu0) [ (p_x(i,j,k) - p_x(i,j+1,k)) / Ly_j + (p_y(i+1,j,k) - p_y(i,j,k)) / Lx_i ]
// and the edges leaving node (i, j, k):
//   (Kp)_x = Lx_i [ F_z(i,j,k) - F_z(i,j-1,k) - F_y(i,j,k) + F_y(i,j,k-1) ]
//   (Kp)_y = Ly_j [ F_x(i,j,k) - F_x(i,j,k-1) - F_z(i,j,k) + F_z(i-1,j,k) ]
//   (Kp)_z = Lz_k [ F_y(i,j,k) - F_y(i-1,j,k) - F_x(i,j,k) + F_x(i,j-1,k) ]
// Edges in the boundary (n x e = 0, Eq. (bc)) are held at zero.
//
// Tiling: a CTA owns a TX x TY column of nodes and marches a chunk of z
// planes.  Plane k and k+1 of the input vector (with a one-node halo) live in
// shared memory; the faces of plane k are computed once into shared memory;
// the faces of plane k-1 that an edge needs stay in registers.
#pragma once

#include <cuda.h>

#include "tem_internal.h"

namespace tem {

// ---------------------------------------------------------------- bounds-checked build
// Built with -DTEM_CHECK_BOUNDS, the hot kernels check every global index (and the alignment of
// every TMA box) before the access.  A failing check records the first (site, index) in a
// device word and skips the access instead of faulting; Batch::solve and the server report it.
// Without the macro every check is the constant true and compiles away.
#ifdef TEM_CHECK_BOUNDS
static __device__ unsigned long long g_tem_fault = 0ull;
__device__ __forceinline__ bool index_ok(int64_t idx, int64_t n, int site) {
  if (idx >= 0 && idx < n) return true;
  atomicCAS(&g_tem_fault, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xffffffffffffull));
  return false;
}
#define TEM_CHECK(idx, n, site) ::tem::index_ok((int64_t)(idx), (int64_t)(n), (site))
// Read and clear the record (0: no failed check); host side, synchronises the stream.
static inline unsigned long long take_bounds_fault(cudaStream_t st) {
  unsigned long long v = 0ull;
  const unsigned long long z = 0ull;
  cudaMemcpyFromSymbolAsync(&v, g_tem_fault, sizeof(v), 0, cudaMemcpyDeviceToHost, st);
  cudaMemcpyToSymbolAsync(g_tem_fault, &z, sizeof(z), 0, cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  return v;
}
#else
#define TEM_CHECK(idx, n, site) true
static inline unsigned long long take_bounds_fault(cudaStream_t) { return 0ull; }
#endif

// ---------------------------------------------------------------- complex
template <class T> struct C2 {
  T re, im;
  __host__ __device__ C2() {}
  __host__ __device__ C2(T r, T i) : re(r), im(i) {}
};
template <class T> __device__ __forceinline__ C2<T> operator+(C2<T> a, C2<T> b) { return C2<T>(a.re + b.re, a.im + b.im); }
template <class T> __device__ __forceinline__ C2<T> operator-(C2<T> a, C2<T> b) { return C2<T>(a.re - b.re, a.im - b.im); }
template <class T> __device__ __forceinline__ C2<T> operator*(T s, C2<T> a) { return C2<T>(s * a.re, s * a.im); }
template <class T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> __device__ __forceinline__ C2<T> cdiv(C2<T> a, C2<T> b) {
  T d = T(1) / (b.re * b.re + b.im * b.im);
  return C2<T>((a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d);
}
template <class T> __device__ __forceinline__ C2<T> czero() { return C2<T>(T(0), T(0)); }

template <class T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

template <class T> __device__ __forceinline__ C2<T> ld(const void* base, int64_t idx) {
  typedef typename Vec2<T>::type V;
  V v = __ldg(reinterpret_cast<const V*>(base) + idx);
  return C2<T>(v.x, v.y);
}
template <class T> __device__ __forceinline__ void st(void* base, int64_t idx, C2<T> a) {
  typedef typename Vec2<T>::type V;
  V v; v.x = a.re; v.y = a.im;
  reinterpret_cast<V*>(base)[idx] = v;
}

// 1-D geometry accessors in the working precision
template <class T> struct Geo;
template <> struct Geo<double> {
  const double *Lx, *Ly, *Lz, *Sx, *Sy, *Sz, *Rx, *Ry, *Rz, *Me, *Wn, *dK;
  __device__ Geo(const GridView& g)
      : Lx(g.Lx), Ly(g.Ly), Lz(g.Lz), Sx(g.Sx), Sy(g.Sy), Sz(g.Sz), Rx(g.Rx), Ry(g.Ry), Rz(g.Rz), Me(g.Me), Wn(g.Wn),
        dK(g.dK) {}
};
template <> struct Geo<float> {
  const float *Lx, *Ly, *Lz, *Sx, *Sy, *Sz, *Rx, *Ry, *Rz, *Me, *Wn, *dK;
  __device__ Geo(const GridView& g)
      : Lx(g.Lxf), Ly(g.Lyf), Lz(g.Lzf), Sx(g.Sxf), Sy(g.Syf), Sz(g.Szf), Rx(g.Rxf), Ry(g.Ryf), Rz(g.Rzf),
        Me(g.Mef), Wn(g.Wnf), dK(g.dKf) {}
};

// Diagonal of K at edge (c, i, j, k) (valid, non-boundary edges only):
//   x: Lx_i/mu0 [ Sz_k (1/Ly_j + 1/Ly_{j-1}) + Sy_j (1/Lz_k + 1/Lz_{k-1}) ]   and cyclically.
template <class T>
__device__ __forceinline__ T diagK(const Geo<T>& G, int c, int i, int j, int k) {
  const T inv_mu0 = T(1.0 / TEM_MU0);
  if (c == 0) return G.Lx[i] * inv_mu0 * (G.Sz[k] * (G.Ry[j] + G.Ry[j - 1]) + G.Sy[j] * (G.Rz[k] + G.Rz[k - 1]));
  if (c == 1) return G.Ly[j] * inv_mu0 * (G.Sz[k] * (G.Rx[i] + G.Rx[i - 1]) + G.Sx[i] * (G.Rz[k] + G.Rz[k - 1]));
  return G.Lz[k] * inv_mu0 * (G.Sx[i] * (G.Ry[j] + G.Ry[j - 1]) + G.Sy[j] * (G.Rx[i] + G.Rx[i - 1]));
}

// Is edge (c, i, j, k) an unknown (not in the boundary, not padding)?
__device__ __forceinline__ bool edge_valid(int c, int i, int j, int k) {
  return c == 0 ? (j > 0 && k > 0) : (c == 1 ? (i > 0 && k > 0) : (i > 0 && j > 0));
}

// ------------------------------------------------------- deterministic reductions
// Each CTA writes its partial sums to part[slot * stride + local_block]; the last
// CTA of the slot to finish (counted with an atomic ticket) sums them in block
// order, so the result does not depend on scheduling.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
  // warp shuffle, then one value per warp through shared memory, in fixed order
  for (int q = 0; q < NV; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
    for (int q = 0; q < NV; ++q) sh[warp * NV + q] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += sh[w * NV + q];
      v[q] = s;
    }
  }
}

// Returns true in thread 0 of the last CTA of the slot, after which part[] of
// the slot is complete and visible.
template <int NV>
__device__ __forceinline__ bool publish_partial(const double (&v)[NV], double* part, unsigned* ticket,
                                                int nblk, int lb) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NV; ++q) part[(int64_t)lb * NV + q] = v[q];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == (unsigned)nblk - 1u);
    if (last) {
      *ticket = 0u;
      __threadfence();
    }
  }
  __syncthreads();
  return last;
}

// Sum the slot's partials with the whole CTA: thread t adds blocks t, t+NT, ...
// in order, then the fixed shuffle tree; the result lands in thread 0.
template <int NV, int NTH>
__device__ __forceinline__ void sum_partials(const double* part, int nblk, double (&out)[NV], double* sh) {
  for (int q = 0; q < NV; ++q) out[q] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += NTH)
    for (int q = 0; q < NV; ++q) out[q] += __ldcg(part + (int64_t)b * NV + q);
  block_sum<NV, NTH>(out, sh);
}

// ------------------------------------------------------------- stencil core
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int PX = TX + 2;   // plane tile with halo (-1 .. TX)
constexpr int PY = TY + 2;
constexpr int FX = TX + 1;   // face tile (-1 .. TX-1)
constexpr int FY = TY + 1;

constexpr int ZMAX = 64;     // longest z chunk of a stencil CTA

// The CTA's slice of the x and y geometry, staged once: x for i = i0-1 .. i0+TX, y for
// j = j0-1 .. j0+TY (zero outside the grid).  z values are uniform over a plane and are
// read as broadcasts.
template <class T>
struct TileGeo {
  T Lx[PX], Rx[PX], Sx[PX];
  T Ly[PY], Ry[PY], Sy[PY];
};

template <class T>
struct StencilSmem {
  C2<T> P[2][3][PY][PX];
  C2<T> F[3][FY][FX];
  TileGeo<T> geo;
  double red[NT / 32 * 4];
};

template <class T>
__device__ __forceinline__ void stage_geometry(TileGeo<T>& tg, const Geo<T>& G, const GridView& g,
                                               int i0, int j0, int k0, int k1) {
  for (int t = threadIdx.x; t < PX; t += NT) {
    const int i = i0 - 1 + t;
    const bool in = i >= 0 && i < g.nx;
    tg.Lx[t] = in ? G.Lx[i] : T(0);
    tg.Rx[t] = in ? G.Rx[i] : T(0);
    tg.Sx[t] = in ? G.Sx[i] : T(0);
  }
  for (int t = threadIdx.x; t < PY; t += NT) {
    const int j = j0 - 1 + t;
    const bool in = j >= 0 && j < g.ny;
    tg.Ly[t] = in ? G.Ly[j] : T(0);
    tg.Ry[t] = in ? G.Ry[j] : T(0);
    tg.Sy[t] = in ? G.Sy[j] : T(0);
  }
}

// Load plane k of the input into buffer b through the policy's point loader.  Each thread
// owns ceil(3 PY PX / NT) entries; all of its loads are issued before any shared store.
constexpr int LPT = (3 * PY * PX + NT - 1) / NT;
template <class T, class Pol>
__device__ __forceinline__ void load_plane(StencilSmem<T>& sm, int b, int k, int i0, int j0,
                                           const GridView& g, Pol& pol, bool own_plane) {
  C2<T> v[LPT];
  const bool kin = k >= 0 && k < g.nz;
#pragma unroll
  for (int u = 0; u < LPT; ++u) {
    const int t = threadIdx.x + u * NT;
    v[u] = czero<T>();
    if (t < 3 * PY * PX && kin) {
      const int c = t / (PY * PX);
      const int r = t - c * (PY * PX);
      const int jj = r / PX, ii = r - jj * PX;
      const int i = i0 - 1 + ii, j = j0 - 1 + jj;
      if (i >= 0 && i < g.nx && j >= 0 && j < g.ny) {
        const int64_t idx = (int64_t)c * g.ncomp + i + (int64_t)g.nx * (j + (int64_t)g.ny * k);
        const bool own = own_plane && ii >= 1 && ii <= TX && jj >= 1 && jj <= TY;
        v[u] = pol.load(c, i, j, k, idx, own);
      }
    }
  }
  C2<T>* P = &sm.P[b][0][0][0];
#pragma unroll
  for (int u = 0; u < LPT; ++u) {
    const int t = threadIdx.x + u * NT;
    if (t < 3 * PY * PX) P[t] = v[u];
  }
}

// Faces of plane k (buffer bk) using plane k+1 (buffer bk1), for the tile plus its -1 halo;
// rLz = 1/Lz_k, sZ = Sz_k / mu0.
template <class T>
__device__ __forceinline__ void compute_faces(StencilSmem<T>& sm, int bk, int bk1, T rLz, T sZ, int i0, int j0,
                                              const GridView& g) {
  const T inv_mu0 = T(1.0 / TEM_MU0);
  const TileGeo<T>& tg = sm.geo;
  for (int t = threadIdx.x; t < FY * FX; t += NT) {
    const int jj = t / FX, ii = t - jj * FX;
    const int i = i0 - 1 + ii, j = j0 - 1 + jj;
    C2<T> fx = czero<T>(), fy = czero<T>(), fz = czero<T>();
    if (i >= 0 && i < g.nx && j >= 0 && j < g.ny) {
      const T rLx = tg.Rx[ii], rLy = tg.Ry[jj];
      // plane-k values around (ii, jj)
      const C2<T> px = sm.P[bk][0][jj][ii], py = sm.P[bk][1][jj][ii], pz = sm.P[bk][2][jj][ii];
      const C2<T> pz_j1 = sm.P[bk][2][jj + 1][ii];
      const C2<T> pz_i1 = sm.P[bk][2][jj][ii + 1];
      const C2<T> px_j1 = sm.P[bk][0][jj + 1][ii];
      const C2<T> py_i1 = sm.P[bk][1][jj][ii + 1];
      const C2<T> px_k1 = sm.P[bk1][0][jj][ii];
      const C2<T> py_k1 = sm.P[bk1][1][jj][ii];
      fx = (tg.Sx[ii] * inv_mu0) * (rLz * (py - py_k1) + rLy * (pz_j1 - pz));
      fy = (tg.Sy[jj] * inv_mu0) * (rLx * (pz - pz_i1) + rLz * (px_k1 - px));
      fz = sZ * (rLy * (px - px_j1) + rLx * (py_i1 - py));
    }
    sm.F[0][jj][ii] = fx;
    sm.F[1][jj][ii] = fy;
    sm.F[2][jj][ii] = fz;
  }
}

// Own faces F_x, F_y of plane k for the thread at (ii, jj), straight from the planes.
template <class T>
__device__ __forceinline__ void own_faces_xy(const StencilSmem<T>& sm, int bk, int bk1, int k, T rLz, int i, int j,
                                             int ii, int jj, const GridView& g, C2<T>& fx, C2<T>& fy) {
  fx = czero<T>();
  fy = czero<T>();
  if (k < 0 || k >= g.nz || i >= g.nx || j >= g.ny) return;
  const T inv_mu0 = T(1.0 / TEM_MU0);
  const TileGeo<T>& tg = sm.geo;
  const T rLx = tg.Rx[ii], rLy = tg.Ry[jj];
  const C2<T> px = sm.P[bk][0][jj][ii], py = sm.P[bk][1][jj][ii], pz = sm.P[bk][2][jj][ii];
  fx = (tg.Sx[ii] * inv_mu0) * (rLz * (py - sm.P[bk1][1][jj][ii]) + rLy * (sm.P[bk][2][jj + 1][ii] - pz));
  fy = (tg.Sy[jj] * inv_mu0) * (rLx * (pz - sm.P[bk][2][jj][ii + 1]) + rLz * (sm.P[bk1][0][jj][ii] - px));
}

// The z-marching stencil: for every own valid edge of planes [k0, k1) calls
// pol.edge(c, idx, i, j, k, p_e, (Kp)_e), after pol.node(n, i, j, k, tg, ii, jj, kz) for its
// node; invalid own edges get pol.edge_invalid(idx).
template <class T, class Pol>
__device__ __forceinline__ void stencil_march(StencilSmem<T>& sm, const GridView& g, Pol& pol,
                                              int i0, int j0, int k0, int k1) {
  const Geo<T> G(g);
  stage_geometry<T>(sm.geo, G, g, i0, j0, k0, k1);
  const int a = threadIdx.x % TX, b = threadIdx.x / TX;
  const int i = i0 + a, j = j0 + b;
  const int ii = a + 1, jj = b + 1;
  // prologue: planes k0-1 (buffer 0) and k0 (buffer 1)
  load_plane<T>(sm, 0, k0 - 1, i0, j0, g, pol, false);
  load_plane<T>(sm, 1, k0, i0, j0, g, pol, true);
  __syncthreads();
  C2<T> fxm, fym;  // F_x, F_y of plane k-1 at (i, j)
  own_faces_xy<T>(sm, 0, 1, k0 - 1, k0 > 0 ? G.Rz[k0 - 1] : T(0), i, j, ii, jj, g, fxm, fym);
  if (i < g.nx && j < g.ny)
    pol.prev_plane(i + (int64_t)g.nx * (j + (int64_t)g.ny * (k0 - 1)), i, j, k0 - 1, sm.P[0][2][jj][ii],
                   k0 > 0 ? G.Rz[k0 - 1] : T(0));
  int bk = 1;  // buffer of plane k
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const int bk1 = bk ^ 1;
    const T lz = G.Lz[k], rz = G.Rz[k], szm = G.Sz[k] * T(1.0 / TEM_MU0);
    __syncthreads();  // buffer bk1 (plane k-1) and F are free
    load_plane<T>(sm, bk1, k + 1, i0, j0, g, pol, k + 1 < k1);
    if (i < g.nx && j < g.ny) pol.prefetch(i + (int64_t)g.nx * (j + (int64_t)g.ny * k), i, j, k);
    __syncthreads();
    compute_faces<T>(sm, bk, bk1, rz, szm, i0, j0, g);
    __syncthreads();
    if (i < g.nx && j < g.ny) {
      const TileGeo<T>& tg = sm.geo;
      const int64_t base = i + (int64_t)g.nx * (j + (int64_t)g.ny * k);
      pol.node(base, i, j, k, tg.Rx[ii], tg.Ry[jj], rz);
      const C2<T> fx = sm.F[0][jj][ii], fy = sm.F[1][jj][ii], fz = sm.F[2][jj][ii];
      // x-edge
      if (edge_valid(0, i, j, k)) {
        const C2<T> kp = tg.Lx[ii] * ((fz - sm.F[2][jj - 1][ii]) - (fy - fym));
        pol.edge(0, base, i, j, k, sm.P[bk][0][jj][ii], kp);
      } else {
        pol.edge_invalid(base);
      }
      if (edge_valid(1, i, j, k)) {
        const C2<T> kp = tg.Ly[jj] * ((fx - fxm) - (fz - sm.F[2][jj][ii - 1]));
        pol.edge(1, g.ncomp + base, i, j, k, sm.P[bk][1][jj][ii], kp);
      } else {
        pol.edge_invalid(g.ncomp + base);
      }
      if (edge_valid(2, i, j, k)) {
        const C2<T> kp = lz * ((fy - sm.F[1][jj][ii - 1]) - (fx - sm.F[0][jj - 1][ii]));
        pol.edge(2, 2 * g.ncomp + base, i, j, k, sm.P[bk][2][jj][ii], kp);
      } else {
        pol.edge_invalid(2 * g.ncomp + base);
      }
      pol.node_end(base, i, j, k, sm.P[bk][0][jj][ii - 1], sm.P[bk][1][jj - 1][ii], sm.P[bk][2][jj][ii],
                   tg.Rx[ii - 1], tg.Ry[jj - 1], tg.Rx[ii], tg.Ry[jj], rz);
      fxm = fx;
      fym = fy;
    }
    bk = bk1;
  }
}

// --------------------------------------------------------------- slot plumbing
// Block lists: CTA -> (slot, the CTA's block index within the slot).  The lists interleave the
// slots block by block (see build_block_maps), and a slot's arithmetic depends only on its own
// block index, never on its position in the list.  In FP32, the stencil and update lists hold
// first the blocks of the slots that take the TMA / 16-byte kernels (even nx), then the others;
// each part is its own launch, so a slot runs the same kernels whatever else is in the batch.
struct BatchArgs {
  const SlotDesc* slots;
  SlotScalars* sc;
  const int2* blk2slot;      // stencil / residual launch
  const int2* ublk2slot;     // update launch
  const int2* nblk2slot;     // nodal launch
  const CUtensorMap* tmaps;  // [slot][7] tile maps of the FP32 stencil pass (or NULL)
  double* part;              // [slot][part_stride] partial sums
  unsigned* ticket;          // [slot]
  int* n_active;             // slots armed or iterating
  int part_stride;           // doubles per slot in part
};

__device__ __forceinline__ void tile_of(const SlotDesc& d, int lb, int nz, int& i0, int& j0, int& k0, int& k1) {
  const int zchunk = d.zchunk;
  const int tx = lb % d.tiles_x;
  const int r = lb / d.tiles_x;
  const int ty = r % d.tiles_y;
  const int zc = r / d.tiles_y;
  i0 = tx * TX;
  j0 = ty * TY;
  k0 = zc * zchunk;
  k1 = min(k0 + zchunk, nz);
}

// ---------------------------------------------------------- the preconditioner
// Jacobi on the edges plus a correction in the gradient (near-null) space of K
// (the auxiliary-space idea of Hiptmair & Xu 2007):
//     z = D^{-1} r + G psi,   psi = D_n^{-1} G^T r,
//     D = diag(K) - xi M,     D_n = diag(G^T A G) = -xi diag(G^T M G) = -xi W,
// with G the gradient of interior-node potentials ((G phi)_e = (phi_end - phi_start) / L_e).
// Both terms are complex symmetric, so COCG applies.  The iteration keeps every
// direction split as p = a + G b (a on edges, b on nodes), so that
//     A p = (K - xi M) a - xi M G b          (K G = 0 exactly, since curl grad = 0),
// and K never acts on the large gradient part: in FP32 the rounding of a large
// gradient would otherwise not be annihilated by K.
template <class T>
__device__ __forceinline__ C2<T> jacobi_D(const Geo<T>& G, int, int, int, int, int64_t idx, C2<T> xi) {
  return C2<T>(G.dK[idx], T(0)) - (G.Me[idx] * xi);
}

// (G b)_e for edge (c, i, j, k) from nodal values; nodes at index n (boundary) hold 0.
template <class T>
__device__ __forceinline__ C2<T> grad_edge(const Geo<T>& G, const GridView& g, int c, int i, int j, int k,
                                           int64_t n0, C2<T> b0, const void* bv, C2<T> beta, const void* bold,
                                           const void* psi, bool use_beta) {
  int64_t n1;
  bool in;
  T rl;
  if (c == 0) { in = i + 1 < g.nx; n1 = n0 + 1; rl = G.Rx[i]; }
  else if (c == 1) { in = j + 1 < g.ny; n1 = n0 + g.nx; rl = G.Ry[j]; }
  else { in = k + 1 < g.nz; n1 = n0 + (int64_t)g.nx * g.ny; rl = G.Rz[k]; }
  C2<T> b1 = czero<T>();
  if (in) {
    if (bv) b1 = ld<T>(bv, n1);
    else {
      b1 = ld<T>(psi, n1);
      if (use_beta) b1 = b1 + cmul(beta, ld<T>(bold, n1));
    }
  }
  return rl * (b1 - b0);
}

// ---------------------- pass A: a <- w + beta a, b <- psi + beta b, q <- A (a + G b), (p, q)
template <class T>
struct CocgStencilPol {
  typedef typename Vec2<T>::type V;
  const V* __restrict__ w; const V* __restrict__ aold; V* __restrict__ anew; V* __restrict__ q;
  const V* __restrict__ psi; const V* __restrict__ bold; V* __restrict__ bnew;  // nodal part (NULL: Jacobi)
  const T* __restrict__ Me;
  C2<T> beta; bool use_beta;
  C2<T> xi;
  const GridView* g;
  C2<T> acc;
  V* __restrict__ gpo;   // G^T M p per own interior node (NULL with Jacobi only)
  // prefetched nodal values: own node, +x, +y, +z, -x, -y neighbours, and masses
  C2<T> pb[6], po[6];
  T me[3], mxm, mym;
  C2<T> gb[3], pc[3];
  C2<T> b0;
  // the own column one plane below: a_z, b, M_z and 1/Lz there
  C2<T> az_prev, b_prev;
  T mz_prev, rz_prev;
  __device__ CocgStencilPol(const GridView& gv) : g(&gv) {}
  __device__ static C2<T> L(const V* p, int64_t i) { const V v = __ldg(p + i); return C2<T>(v.x, v.y); }
  __device__ static void S(V* p, int64_t i, C2<T> a) { V v; v.x = a.re; v.y = a.im; p[i] = v; }
  __device__ C2<T> bnode(int64_t n) const {
    const C2<T> v = L(psi, n);
    return use_beta ? v + cmul(beta, L(bold, n)) : v;
  }
  __device__ C2<T> load(int c, int i, int j, int k, int64_t idx, bool own) {
    if (!edge_valid(c, i, j, k)) return czero<T>();  // boundary: a stays 0 (buffers start zeroed)
    C2<T> v = L(w, idx);
    if (use_beta) v = v + cmul(beta, L(aold, idx));
    if (own) S(anew, idx, v);
    return v;
  }
  // the plane below the chunk: a_z there comes from the shared plane, b and M_z from memory
  __device__ void prev_plane(int64_t n, int, int, int k, C2<T> az, T rzp) {
    az_prev = az;
    rz_prev = rzp;
    b_prev = czero<T>();
    mz_prev = T(0);
    if (!psi || k < 0) return;
    b_prev = bnode(n);
    mz_prev = __ldg(Me + 2 * g->ncomp + n);
  }
  // issue the loads the edges of node n will need, before the face phase
  __device__ void prefetch(int64_t n, int i, int j, int k) {
    const int64_t nc = g->ncomp;
    me[0] = __ldg(Me + n);
    me[1] = __ldg(Me + nc + n);
    me[2] = __ldg(Me + 2 * nc + n);
    if (!psi) return;
    const bool interior = i > 0 && j > 0 && k > 0;
    mxm = interior ? __ldg(Me + n - 1) : T(0);
    mym = interior ? __ldg(Me + nc + n - g->nx) : T(0);
    const int64_t nb[6] = {n, n + 1, n + g->nx, n + (int64_t)g->nx * g->ny, n - 1, n - g->nx};
    const bool in[6] = {true, i + 1 < g->nx, j + 1 < g->ny, k + 1 < g->nz, interior, interior};
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      pb[u] = in[u] ? L(psi, nb[u]) : czero<T>();
      po[u] = (in[u] && use_beta) ? L(bold, nb[u]) : czero<T>();
    }
  }
  __device__ void node(int64_t n, int, int, int, T rx, T ry, T rz) {   // once per own node
    pc[0] = pc[1] = pc[2] = czero<T>();
    if (!psi) return;
    C2<T> b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = use_beta ? pb[u] + cmul(beta, po[u]) : pb[u];
    b0 = b[0];
    S(bnew, n, b0);
    gb[0] = rx * (b[1] - b[0]);
    gb[1] = ry * (b[2] - b[0]);
    gb[2] = rz * (b[3] - b[0]);
  }
  __device__ void edge(int c, int64_t idx, int, int, int, C2<T> a, C2<T> ka) {
    const C2<T> p = psi ? a + gb[c] : a;
    pc[c] = p;
    const C2<T> qv = ka - cmul(xi, me[c] * p);
    S(q, idx, qv);
    acc = acc + cmul(p, qv);
  }
  // (G^T M p)_n from the six edges at node n: +M p / L on the three arriving edges,
  // -M p / L on the three leaving ones; then roll the column state up one plane
  __device__ void node_end(int64_t n, int i, int j, int k, C2<T> ax_m, C2<T> ay_m, C2<T> az_own,
                           T rx_m, T ry_m, T rx, T ry, T rz) {
    if (psi) {
      if (i > 0 && j > 0 && k > 0) {
        const C2<T> bxm = use_beta ? pb[4] + cmul(beta, po[4]) : pb[4];
        const C2<T> bym = use_beta ? pb[5] + cmul(beta, po[5]) : pb[5];
        const C2<T> pxm = ax_m + rx_m * (b0 - bxm);
        const C2<T> pym = ay_m + ry_m * (b0 - bym);
        const C2<T> pzm = az_prev + rz_prev * (b0 - b_prev);
        const C2<T> v = (rx_m * mxm) * pxm + (ry_m * mym) * pym + (rz_prev * mz_prev) * pzm -
                        (rx * me[0]) * pc[0] - (ry * me[1]) * pc[1] - (rz * me[2]) * pc[2];
        S(gpo, n, v);
      }
      b_prev = b0;
      mz_prev = me[2];
    }
    az_prev = az_own;
    rz_prev = rz;
  }
  __device__ void edge_invalid(int64_t idx) { S(q, idx, czero<T>()); }
};

// FP32: at least 3 CTAs (24 warps) per SM; FP64 keeps its registers (it is bound by FP64 issue)
template <class T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 2) k_cocg_stencil(BatchArgs A) {
  __shared__ StencilSmem<T> sm;
  const int2 bm = A.blk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  if (!S->active) return;
  const SlotDesc& d = A.slots[slot];
  int i0, j0, k0, k1;
  tile_of(d, lb, d.g.nz, i0, j0, k0, k1);
  CocgStencilPol<T> pol(d.g);
  typedef typename Vec2<T>::type V;
  pol.w = static_cast<const V*>(d.w);
  pol.aold = static_cast<const V*>(S->parity ? d.a1 : d.a0);
  pol.anew = static_cast<V*>(S->parity ? d.a0 : d.a1);
  pol.psi = d.nodal ? static_cast<const V*>(d.psi) : nullptr;
  pol.bold = static_cast<const V*>(S->parity ? d.b1 : d.b0);
  pol.bnew = static_cast<V*>(S->parity ? d.b0 : d.b1);
  pol.q = static_cast<V*>(d.q);
  pol.gpo = static_cast<V*>(d.gp);
  pol.Me = Geo<T>(d.g).Me;
  pol.beta = C2<T>(T(S->beta_re), T(S->beta_im));
  pol.use_beta = !(S->beta_re == 0.0 && S->beta_im == 0.0);
  pol.xi = C2<T>(T(d.xi_re), T(d.xi_im));
  pol.acc = czero<T>();
  stencil_march<T>(sm, d.g, pol, i0, j0, k0, k1);
  double v[2] = {double(pol.acc.re), double(pol.acc.im)};
  block_sum<2, NT>(v, sm.red);
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<2>(v, part, A.ticket + slot, d.nblk_stencil, lb)) {
    double tot[2];
    sum_partials<2, NT>(part, d.nblk_stencil, tot, sm.red);
    if (threadIdx.x != 0) return;
    // alpha = rho / (p, A p)
    const double den = tot[0] * tot[0] + tot[1] * tot[1];
    if (!(den > 0.0) || !isfinite(den)) {
      S->status = TEM_EBREAKDOWN;
      S->active = 0;
      S->total_iters += S->iters;
      atomicSub(A.n_active, 1);
    } else {
      S->alpha_re = (S->rho_re * tot[0] + S->rho_im * tot[1]) / den;
      S->alpha_im = (S->rho_im * tot[0] - S->rho_re * tot[1]) / den;
    }
  }
}

// --------------------------- pass A, FP32, asynchronously pipelined through shared memory
// The same arithmetic as k_cocg_stencil with the raw inputs of each z plane (w, a_old on the
// edges; psi, b_old on the nodes; tile plus one-node halo) streamed into a shared ring of
// TEM_PIPE_STAGES planes by cp.async, up to that many planes ahead of the compute.  a = w + beta a_old and
// b = psi + beta b_old are formed in shared memory for planes k and k+1, so every gradient
// (G b) and every (G^T M p) term reads shared memory.  Out-of-grid halo entries are
// zero-filled by the copies; boundary entries are stored as zeros.
#ifndef TEM_PIPE_STAGES
#define TEM_PIPE_STAGES 2          // raw planes in the shared ring (>= 2; 2 and 3 measured within 1 %)
#endif
#ifndef TEM_PIPE_MIN_CTAS
#define TEM_PIPE_MIN_CTAS 2        // occupancy target of the pipelined stencil (CTAs per SM)
#endif
namespace pipe {
constexpr int NA = 8;              // staged arrays: w[3], a_old[3], psi, b_old
constexpr int NS = TEM_PIPE_STAGES;
constexpr int PLANE = PY * PX;     // entries of one component plane (with halo)
struct Smem {
  float2 stage[NS][NA][PLANE];     // raw planes
  float2 P[2][4][PLANE];           // a (3 components) and b for planes k, k+1
  float2 F[3][FY][FX];             // faces of plane k
  TileGeo<float> geo;
  double red[NT / 32 * 4];
};
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = pred ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void wait_pending() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
}  // namespace pipe

struct PipeArgs {
  const float2* w; const float2* aold; const float2* psi; const float2* bold;
  bool use_beta, nodal;
};

// The halo positions a thread copies and forms are the same on every plane: up to
// PPT = ceil(PLANE / NT) positions, with their shared index, in-plane offset i + nx j
// (or -1 outside the grid) and whether they are own (interior of the tile).
constexpr int PPT = (pipe::PLANE + NT - 1) / NT;
struct PipePos {
  int r[PPT];
  int64_t off[PPT];
  bool own[PPT];
};

__device__ __forceinline__ void pipe_positions(PipePos& pp, int i0, int j0, const GridView& g) {
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int r = threadIdx.x + u * NT;
    pp.r[u] = r < pipe::PLANE ? r : -1;
    const int jj = r / PX, ii = r - jj * PX;
    const int i = i0 - 1 + ii, j = j0 - 1 + jj;
    const bool in = r < pipe::PLANE && i >= 0 && i < g.nx && j >= 0 && j < g.ny;
    pp.off[u] = in ? i + (int64_t)g.nx * j : -1;
    pp.own[u] = in && ii >= 1 && ii <= TX && jj >= 1 && jj <= TY;
  }
}

// issue the copies of plane k into stage st; planes past klast are skipped
__device__ __forceinline__ void pipe_issue(pipe::Smem& sm, const PipePos& pp, int st, int k, int klast,
                                           const GridView& g, const PipeArgs& pa) {
  if (k > klast) return;
  const bool kin = k >= 0 && k < g.nz;
  const int64_t gk = (int64_t)g.nx * g.ny * k;
  const int64_t nc = g.ncomp;
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int r = pp.r[u];
    if (r < 0) continue;
    const bool in = kin && pp.off[u] >= 0;
    const int64_t n = in ? gk + pp.off[u] : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pipe::cp_async8(&sm.stage[st][c][r], in ? pa.w + c * nc + n : pa.w, in);
      const bool ua = in && pa.use_beta;
      pipe::cp_async8(&sm.stage[st][3 + c][r], ua ? pa.aold + c * nc + n : pa.w, ua);
    }
    const bool un = in && pa.nodal;
    pipe::cp_async8(&sm.stage[st][6][r], un ? pa.psi + n : pa.w, un);
    const bool ub = un && pa.use_beta;
    pipe::cp_async8(&sm.stage[st][7][r], ub ? pa.bold + n : pa.w, ub);
  }
}

// P[b] <- plane k from stage st; own entries of a and b are written to anew / bnew
__device__ __forceinline__ void pipe_form(pipe::Smem& sm, const PipePos& pp, int b, int st, int k,
                                          const GridView& g, C2<float> beta, bool own_plane, float2* anew,
                                          float2* bnew) {
  const int64_t gk = (int64_t)g.nx * g.ny * k;
  const int64_t nc = g.ncomp;
#pragma unroll
  for (int u = 0; u < PPT; ++u) {
    const int r = pp.r[u];
    if (r < 0) continue;
    const bool own = own_plane && pp.own[u];
    const int64_t n = gk + pp.off[u];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float2 v = sm.stage[st][c < 3 ? c : 6][r];
      const float2 o = sm.stage[st][c < 3 ? 3 + c : 7][r];
      v.x += beta.re * o.x - beta.im * o.y;
      v.y += beta.re * o.y + beta.im * o.x;
      sm.P[b][c][r] = v;
      if (own) {
        if (c < 3) {
          if (TEM_CHECK(c * nc + n, 3 * nc, 1)) anew[c * nc + n] = v;
        } else if (bnew && TEM_CHECK(n, nc, 2)) {
          bnew[n] = v;
        }
      }
    }
  }
}

__device__ __forceinline__ void pipe_faces(pipe::Smem& sm, int bk, int bk1, float rLz, float sZ, int i0, int j0,
                                           const GridView& g) {
  const float inv_mu0 = float(1.0 / TEM_MU0);
  const TileGeo<float>& tg = sm.geo;
  for (int t = threadIdx.x; t < FY * FX; t += NT) {
    const int jj = t / FX, ii = t - jj * FX;
    const int i = i0 - 1 + ii, j = j0 - 1 + jj;
    float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx;
    if (i >= 0 && i < g.nx && j >= 0 && j < g.ny) {
      const int r = jj * PX + ii;
      const float rLx = tg.Rx[ii], rLy = tg.Ry[jj];
      const float2 px = sm.P[bk][0][r], py = sm.P[bk][1][r], pz = sm.P[bk][2][r];
      const float2 pz_j1 = sm.P[bk][2][r + PX], pz_i1 = sm.P[bk][2][r + 1];
      const float2 px_j1 = sm.P[bk][0][r + PX], py_i1 = sm.P[bk][1][r + 1];
      const float2 px_k1 = sm.P[bk1][0][r], py_k1 = sm.P[bk1][1][r];
      const float sx = tg.Sx[ii] * inv_mu0, sy = tg.Sy[jj] * inv_mu0;
      fx.x = sx * (rLz * (py.x - py_k1.x) + rLy * (pz_j1.x - pz.x));
      fx.y = sx * (rLz * (py.y - py_k1.y) + rLy * (pz_j1.y - pz.y));
      fy.x = sy * (rLx * (pz.x - pz_i1.x) + rLz * (px_k1.x - px.x));
      fy.y = sy * (rLx * (pz.y - pz_i1.y) + rLz * (px_k1.y - px.y));
      fz.x = sZ * (rLy * (px.x - px_j1.x) + rLx * (py_i1.x - py.x));
      fz.y = sZ * (rLy * (px.y - px_j1.y) + rLx * (py_i1.y - py.y));
    }
    sm.F[0][jj][ii] = fx;
    sm.F[1][jj][ii] = fy;
    sm.F[2][jj][ii] = fz;
  }
}

static __global__ void __launch_bounds__(NT, TEM_PIPE_MIN_CTAS) k_cocg_stencil_pipe(BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pipe::Smem& sm = *reinterpret_cast<pipe::Smem*>(smem_raw);
  const int2 bm = A.blk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  if (!S->active) return;
  const SlotDesc& d = A.slots[slot];
  const GridView& g = d.g;
  int i0, j0, k0, k1;
  tile_of(d, lb, g.nz, i0, j0, k0, k1);
  PipeArgs pa;
  pa.w = static_cast<const float2*>(d.w);
  pa.aold = static_cast<const float2*>(S->parity ? d.a1 : d.a0);
  pa.psi = static_cast<const float2*>(d.psi);
  pa.bold = static_cast<const float2*>(S->parity ? d.b1 : d.b0);
  pa.use_beta = !(S->beta_re == 0.0 && S->beta_im == 0.0);
  pa.nodal = d.nodal != 0;
  float2* anew = static_cast<float2*>(S->parity ? d.a0 : d.a1);
  float2* bnew = pa.nodal ? static_cast<float2*>(S->parity ? d.b0 : d.b1) : nullptr;
  float2* q = static_cast<float2*>(d.q);
  float2* gpo = static_cast<float2*>(d.gp);
  const C2<float> beta(pa.use_beta ? float(S->beta_re) : 0.f, pa.use_beta ? float(S->beta_im) : 0.f);
  const C2<float> xi(float(d.xi_re), float(d.xi_im));
  const Geo<float> G(g);
  const float* __restrict__ Me = G.Me;
  // stage geometry, start the first three planes
  stage_geometry<float>(sm.geo, G, g, i0, j0, k0, k1);
  PipePos pp;
  pipe_positions(pp, i0, j0, g);
  // plane p lives in stage (p - k0 + 1) mod NS; planes k0-1 .. k1 are needed.  After the
  // prologue and after every round, the planes k+1 .. k+NS-1 are in flight (one group each).
  static_assert(pipe::NS >= 2, "two stages at least");
#pragma unroll
  for (int u = 0; u < pipe::NS; ++u) {
    pipe_issue(sm, pp, u, k0 - 1 + u, k1, g, pa);
    pipe::commit();
  }
  pipe::wait_pending<pipe::NS - 2>();
  __syncthreads();
  pipe_form(sm, pp, 0, 0, k0 - 1, g, beta, false, anew, bnew);
  pipe_form(sm, pp, 1, 1 % pipe::NS, k0, g, beta, true, anew, bnew);
  __syncthreads();
  pipe_issue(sm, pp, 0, k0 - 1 + pipe::NS, k1, g, pa);
  pipe::commit();
  const int a_ = threadIdx.x % TX, b_ = threadIdx.x / TX;
  const int i = i0 + a_, j = j0 + b_;
  const int ii = a_ + 1, jj = b_ + 1, rr0 = jj * PX + ii;
  const bool mine = i < g.nx && j < g.ny;
  const int64_t nc = g.ncomp;
  const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
  const float inv_mu0 = float(1.0 / TEM_MU0);
  // F_x, F_y of plane k0-1 at the own column, and the column state one plane below
  float2 fxm = make_float2(0.f, 0.f), fym = fxm;
  float2 az_prev = sm.P[0][2][rr0], b_prev = sm.P[0][3][rr0];
  float mz_prev = 0.f, rz_prev = 0.f;
  if (mine && k0 > 0) {
    const int km = k0 - 1;
    const float rLz = G.Rz[km];
    const TileGeo<float>& tg = sm.geo;
    const float2 px = sm.P[0][0][rr0], py = sm.P[0][1][rr0], pz = sm.P[0][2][rr0];
    const float sx = tg.Sx[ii] * inv_mu0, syy = tg.Sy[jj] * inv_mu0;
    const float2 pyk = sm.P[1][1][rr0], pxk = sm.P[1][0][rr0];
    const float2 pzj = sm.P[0][2][rr0 + PX], pzi = sm.P[0][2][rr0 + 1];
    fxm.x = sx * (rLz * (py.x - pyk.x) + tg.Ry[jj] * (pzj.x - pz.x));
    fxm.y = sx * (rLz * (py.y - pyk.y) + tg.Ry[jj] * (pzj.y - pz.y));
    fym.x = syy * (tg.Rx[ii] * (pz.x - pzi.x) + rLz * (pxk.x - px.x));
    fym.y = syy * (tg.Rx[ii] * (pz.y - pzi.y) + rLz * (pxk.y - px.y));
    mz_prev = __ldg(Me + 2 * nc + i + sy * j + sz * km);
    rz_prev = rLz;
  }
  C2<float> acc = czero<float>();
  int bk = 1;
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const int bk1 = bk ^ 1;
    const int st_next = (k - k0 + 2) % pipe::NS;      // stage holding plane k+1
    pipe::wait_pending<pipe::NS - 2>();                // plane k+1 has landed
    __syncthreads();
    pipe_form(sm, pp, bk1, st_next, k + 1, g, beta, k + 1 < k1, anew, bnew);
    __syncthreads();
    // plane k + NS goes into plane k's stage, formed last round
    pipe_issue(sm, pp, (k - k0 + 1) % pipe::NS, k + pipe::NS, k1, g, pa);
    pipe::commit();
    const float lz = G.Lz[k], rz = G.Rz[k], szm = G.Sz[k] * inv_mu0;
    const int64_t n = i + sy * j + sz * k;
    const bool interior = mine && i > 0 && j > 0 && k > 0;
    float me0 = 0.f, me1 = 0.f, me2 = 0.f, mxm = 0.f, mym = 0.f;
    if (mine) {
      me0 = __ldg(Me + n);
      me1 = __ldg(Me + nc + n);
      me2 = __ldg(Me + 2 * nc + n);
    }
    if (interior && pa.nodal) {
      mxm = __ldg(Me + n - 1);
      mym = __ldg(Me + nc + n - sy);
    }
    pipe_faces(sm, bk, bk1, rz, szm, i0, j0, g);
    __syncthreads();
    if (mine) {
      const TileGeo<float>& tg = sm.geo;
      const float2 fx = sm.F[0][jj][ii], fy = sm.F[1][jj][ii], fz = sm.F[2][jj][ii];
      const float2 ax = sm.P[bk][0][rr0], ay = sm.P[bk][1][rr0], az = sm.P[bk][2][rr0];
      const float2 b0 = sm.P[bk][3][rr0];
      // (G b) on the three leaving edges
      float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
      if (pa.nodal) {
        const float2 bxp = sm.P[bk][3][rr0 + 1], byp = sm.P[bk][3][rr0 + PX], bzp = sm.P[bk1][3][rr0];
        gx = make_float2(tg.Rx[ii] * (bxp.x - b0.x), tg.Rx[ii] * (bxp.y - b0.y));
        gy = make_float2(tg.Ry[jj] * (byp.x - b0.x), tg.Ry[jj] * (byp.y - b0.y));
        gz = make_float2(rz * (bzp.x - b0.x), rz * (bzp.y - b0.y));
      }
      float2 pc[3] = {make_float2(ax.x + gx.x, ax.y + gx.y), make_float2(ay.x + gy.x, ay.y + gy.y),
                      make_float2(az.x + gz.x, az.y + gz.y)};
      float2 kp[3];
      {
        const float2 fzj = sm.F[2][jj - 1][ii], fzi = sm.F[2][jj][ii - 1];
        const float2 fyi = sm.F[1][jj][ii - 1], fxj = sm.F[0][jj - 1][ii];
        const float lx = tg.Lx[ii], ly = tg.Ly[jj];
        kp[0] = make_float2(lx * ((fz.x - fzj.x) - (fy.x - fym.x)), lx * ((fz.y - fzj.y) - (fy.y - fym.y)));
        kp[1] = make_float2(ly * ((fx.x - fxm.x) - (fz.x - fzi.x)), ly * ((fx.y - fxm.y) - (fz.y - fzi.y)));
        kp[2] = make_float2(lz * ((fy.x - fyi.x) - (fx.x - fxj.x)), lz * ((fy.y - fyi.y) - (fx.y - fxj.y)));
      }
      const float mc[3] = {me0, me1, me2};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 qv = make_float2(0.f, 0.f);
        if (edge_valid(c, i, j, k)) {
          const float mr = mc[c] * pc[c].x, mi = mc[c] * pc[c].y;
          qv.x = kp[c].x - (xi.re * mr - xi.im * mi);
          qv.y = kp[c].y - (xi.re * mi + xi.im * mr);
          acc.re += pc[c].x * qv.x - pc[c].y * qv.y;
          acc.im += pc[c].x * qv.y + pc[c].y * qv.x;
        }
        if (TEM_CHECK(c * nc + n, 3 * nc, 3)) q[c * nc + n] = qv;
      }
      if (interior && pa.nodal) {
        // (G^T M p)_n: +M p / L on the arriving edges, -M p / L on the leaving ones
        const float2 axm = sm.P[bk][0][rr0 - 1], aym = sm.P[bk][1][rr0 - PX];
        const float2 bxm = sm.P[bk][3][rr0 - 1], bym = sm.P[bk][3][rr0 - PX];
        const float rxm = tg.Rx[ii - 1], rym = tg.Ry[jj - 1];
        const float2 pxm = make_float2(axm.x + rxm * (b0.x - bxm.x), axm.y + rxm * (b0.y - bxm.y));
        const float2 pym = make_float2(aym.x + rym * (b0.x - bym.x), aym.y + rym * (b0.y - bym.y));
        const float2 pzm = make_float2(az_prev.x + rz_prev * (b0.x - b_prev.x), az_prev.y + rz_prev * (b0.y - b_prev.y));
        const float cx = rxm * mxm, cy = rym * mym, cz = rz_prev * mz_prev;
        const float ox = tg.Rx[ii] * me0, oy = tg.Ry[jj] * me1, oz = rz * me2;
        float2 v;
        v.x = cx * pxm.x + cy * pym.x + cz * pzm.x - ox * pc[0].x - oy * pc[1].x - oz * pc[2].x;
        v.y = cx * pxm.y + cy * pym.y + cz * pzm.y - ox * pc[0].y - oy * pc[1].y - oz * pc[2].y;
        if (TEM_CHECK(n, nc, 4)) gpo[n] = v;
      }
      fxm = fx;
      fym = fy;
      az_prev = az;
      b_prev = b0;
      mz_prev = me2;
      rz_prev = rz;
    }
    bk = bk1;
  }
  pipe::wait_pending<0>();
  double v[2] = {double(acc.re), double(acc.im)};
  block_sum<2, NT>(v, sm.red);
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<2>(v, part, A.ticket + slot, d.nblk_stencil, lb)) {
    double tot[2];
    sum_partials<2, NT>(part, d.nblk_stencil, tot, sm.red);
    if (threadIdx.x != 0) return;
    const double den = tot[0] * tot[0] + tot[1] * tot[1];
    if (!(den > 0.0) || !isfinite(den)) {
      S->status = TEM_EBREAKDOWN;
      S->active = 0;
      S->total_iters += S->iters;
      atomicSub(A.n_active, 1);
    } else {
      S->alpha_re = (S->rho_re * tot[0] + S->rho_im * tot[1]) / den;
      S->alpha_im = (S->rho_im * tot[0] - S->rho_re * tot[1]) / den;
    }
  }
}

// Launch pass A in FP32 through the pipelined kernel (dynamic shared memory above 48 KB).
static inline cudaError_t launch_stencil_pipe(const BatchArgs& A, int nblk, cudaStream_t st) {
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    const cudaError_t e = cudaFuncSetAttribute(k_cocg_stencil_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(pipe::Smem));
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  k_cocg_stencil_pipe<<<nblk, NT, sizeof(pipe::Smem), st>>>(A);
  return cudaGetLastError();
}

// Resident CTAs per SM of the pipelined stencil (0 on error).
static inline int stencil_pipe_occupancy() {
  int n = 0;
  if (cudaFuncSetAttribute(k_cocg_stencil_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(pipe::Smem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cocg_stencil_pipe, NT, sizeof(pipe::Smem)) != cudaSuccess)
    return 0;
  return n;
}

// Convergence test and the next beta, from rho = (r, z) and rr = ||r||^2 (last CTA only).
__device__ __forceinline__ void finish_iteration(SlotScalars* S, int* n_active, double rho_re, double rho_im,
                                                 double rr) {
  // the update pass of this iteration (number S->iters) left alpha p out of d when it is even
  S->lag = (S->iters & 1) == 0;
  S->lag_par = S->parity;
  S->alpha_prev_re = S->alpha_re;
  S->alpha_prev_im = S->alpha_im;
  S->iters += 1;
  S->rr = rr;
  bool done = false;
  if (!isfinite(rho_re) || !isfinite(rho_im) || !isfinite(rr)) {
    S->status = TEM_EBREAKDOWN;
    done = true;
  } else if (rr <= S->tol2) {
    done = true;  // converged
  } else if (S->iters >= S->max_iter) {
    S->status = TEM_ENOCONV;
    done = true;
  } else if (rr >= S->rr_best && S->iters - S->it_best > S->stall_window) {
    done = true;  // stagnation: end this inner solve; the FP64 outer step restarts from the true residual
    S->stalled = 1;
  } else {
    if (rr < S->rr_best) {
      S->rr_best = rr;
      S->it_best = S->iters;
    }
    const double den = S->rho_re * S->rho_re + S->rho_im * S->rho_im;
    if (!(den > 0.0)) {
      S->status = TEM_EBREAKDOWN;
      done = true;
    } else {
      S->beta_re = (rho_re * S->rho_re + rho_im * S->rho_im) / den;
      S->beta_im = (rho_im * S->rho_re - rho_re * S->rho_im) / den;
      S->rho_re = rho_re;
      S->rho_im = rho_im;
      S->parity ^= 1;
    }
  }
  if (done) {
    S->active = 0;
    S->total_iters += S->iters;
    atomicSub(n_active, 1);
  }
}

// The first beta of an inner solve whose right-hand side is s r (r the true FP64 residual).
// A restart takes beta = 0 (p = z).  A solve that continues the last direction p_prev of the
// previous inner solve (scale s_prev; its last rho, rho_prev, still in S->rho) takes the COCG
// beta of the unscaled quantities, rho / rho_prev, times s / s_prev for the scale of the new
// directions:  beta = (rho_s / rho_prev_s) (s_prev / s),  rho_s = s^2 rho.
__device__ __forceinline__ void start_direction(SlotScalars* S, double rho_re, double rho_im) {
  const double den = S->rho_re * S->rho_re + S->rho_im * S->rho_im;
  if (S->carry_ratio > 0.0 && den > 0.0 && isfinite(den)) {
    const double br = (rho_re * S->rho_re + rho_im * S->rho_im) / den;
    const double bi = (rho_im * S->rho_re - rho_re * S->rho_im) / den;
    S->beta_re = br / S->carry_ratio;
    S->beta_im = bi / S->carry_ratio;
  } else {
    S->beta_re = 0.0;
    S->beta_im = 0.0;
  }
  S->rho_re = rho_re;
  S->rho_im = rho_im;
}

// ---------- pass B: r = D w - alpha q, w = r / D; (r, D^-1 r), ||r||; v += alpha xi G^T M p,
// psi = v / D_n; and, on odd iterations t, the correction of two iterations at once:
//   x += alpha_{t-1} a_{t-1} + alpha_t a_t,  x_n += alpha_{t-1} b_{t-1} + alpha_t b_t
// (both directions are still in the two direction buffers; x starts at 0 when t = 1).  An inner
// solve that ends after an even t leaves alpha_t p_t to the residual pass (SlotScalars::lag).
// A stream over the slot's entries [0, 3n) edges, [3n, 4n) nodes; boundary edges have
// diag(K) = 0 and are left alone.
template <class T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 4 : 2) k_cocg_update(BatchArgs A) {
  __shared__ double red[NT / 32 * 4];
  const int2 bm = A.ublk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  if (!S->active) return;
  const SlotDesc& d = A.slots[slot];
  const GridView& g = d.g;
  const C2<T> alpha(T(S->alpha_re), T(S->alpha_im));
  const C2<T> alpha_prev(T(S->alpha_prev_re), T(S->alpha_prev_im));
  const C2<T> xi(T(d.xi_re), T(d.xi_im));
  const bool odd = (S->iters & 1) != 0;             // this pass adds two terms to the correction
  const bool xzero = S->iters == 1;                 // ... which starts at 0
  const void* a = S->parity ? d.a0 : d.a1;          // the direction written by pass A
  const void* b = S->parity ? d.b0 : d.b1;
  const void* ap = S->parity ? d.a1 : d.a0;         // the direction of the previous iteration
  const void* bp = S->parity ? d.b1 : d.b0;
  typedef typename Vec2<T>::type V;
  const T* __restrict__ dK = Geo<T>(g).dK;
  const T* __restrict__ Me = Geo<T>(g).Me;
  const V* __restrict__ qv = static_cast<const V*>(d.q);
  V* __restrict__ wv = static_cast<V*>(d.w);
  const int64_t ne = 3 * g.ncomp;
  const int64_t n = ne + (d.nodal ? g.ncomp : 0);
  const int64_t per = (n + d.nblk_update - 1) / d.nblk_update;
  const int64_t e0 = (int64_t)lb * per, e1 = min(n, e0 + per);
  if (e1 > e0 && !TEM_CHECK(e1 - 1, n, 11)) return;
  C2<T> rz = czero<T>();
  T rr = T(0);
  const int64_t ee = min(e1, ne);
  constexpr int U = 2;
  for (int64_t base = e0 + threadIdx.x; base < ee; base += (int64_t)NT * U) {
    T dk[U], me[U];
    V qr[U], wr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = base + (int64_t)u * NT;
      if (e < ee) {
        dk[u] = __ldg(dK + e);
        me[u] = __ldg(Me + e);
        qr[u] = __ldg(qv + e);
        wr[u] = wv[e];
      } else {
        dk[u] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = base + (int64_t)u * NT;
      if (dk[u] == T(0)) continue;  // boundary entry (or past the range)
      const C2<T> D = C2<T>(dk[u], T(0)) - (me[u] * xi);
      const C2<T> r = cmul(D, C2<T>(wr[u].x, wr[u].y)) - cmul(alpha, C2<T>(qr[u].x, qr[u].y));
      const C2<T> wn = cdiv(r, D);
      V wo; wo.x = wn.re; wo.y = wn.im;
      wv[e] = wo;
      rz = rz + cmul(r, wn);
      rr += r.re * r.re + r.im * r.im;
    }
  }
  // nodal part: v = cn + xi G^T M d += alpha xi G^T M p;  psi = v / D_n
  // (v is kept in the u buffer: the start pass sets it to cn, so cn is not read here)
  const T* __restrict__ Wn = Geo<T>(g).Wn;
  C2<T> rn = czero<T>();
  for (int64_t e = max(e0, ne) + threadIdx.x; e < e1; e += NT) {
    const int64_t m = e - ne;
    const T wn = __ldg(Wn + m);
    if (wn == T(0)) continue;  // boundary node
    const C2<T> dv = ld<T>(d.u, m) + cmul(alpha, cmul(xi, ld<T>(d.gp, m)));
    st<T>(d.u, m, dv);
    const C2<T> ps = cdiv(dv, wn * C2<T>(-xi.re, -xi.im));
    st<T>(d.psi, m, ps);
    rn = rn + cmul(dv, ps);
  }
  // the correction (odd iterations): boundary entries of both directions are 0, so x stays 0 there
  if (odd) {
    for (int64_t e = e0 + threadIdx.x; e < e1; e += NT) {
      const bool edge = e < ne;
      const int64_t m = edge ? e : e - ne;
      void* xd = edge ? d.x : d.xn;
      C2<T> x = xzero ? czero<T>() : ld<T>(xd, m);
      x = x + cmul(alpha_prev, ld<T>(edge ? ap : bp, m));
      x = x + cmul(alpha, ld<T>(edge ? a : b, m));
      st<T>(xd, m, x);
    }
  }
  rz = rz + rn;
  double v[3] = {double(rz.re), double(rz.im), double(rr)};
  block_sum<3, NT>(v, red);
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<3>(v, part, A.ticket + slot, d.nblk_update, lb)) {
    double tot[3];
    sum_partials<3, NT>(part, d.nblk_update, tot, red);
    if (threadIdx.x != 0) return;
    finish_iteration(S, A.n_active, tot[0], tot[1], tot[2]);
  }
}

// ---------- pass B in FP32, two entries per access (16-byte loads and stores)
// The arithmetic of k_cocg_update<float> on entry pairs (2e, 2e+1) of the slot's flat stream:
// 3 n/2 edge pairs, then n/2 node pairs (n = nx ny nz, even for the slots that use this kernel).
// Each thread keeps U pairs of every input in flight before it computes.
__device__ __forceinline__ void update_edge(float& w_re, float& w_im, float q_re, float q_im, float dk, float me,
                                            C2<float> alpha, float xr, float xim, C2<float>& rz, float& rr) {
  if (dk == 0.f) return;   // boundary entry: w stays as it is (0)
  const C2<float> D(dk - me * xr, -me * xim);
  const C2<float> r = cmul(D, C2<float>(w_re, w_im)) - cmul(alpha, C2<float>(q_re, q_im));
  const C2<float> wn = cdiv(r, D);
  w_re = wn.re;
  w_im = wn.im;
  rz = rz + cmul(r, wn);
  rr += r.re * r.re + r.im * r.im;
}

// v = cn + xi G^T M d (kept in the u buffer; the start pass sets it to cn): v += alpha xi G^T M p
__device__ __forceinline__ void update_node(float& v_re, float& v_im, float& ps_re, float& ps_im, float gp_re,
                                            float gp_im, float wn, C2<float> alpha, C2<float> xi, C2<float>& rn) {
  if (wn == 0.f) return;   // boundary node: v and psi stay 0
  const C2<float> ag = cmul(alpha, cmul(xi, C2<float>(gp_re, gp_im)));
  v_re += ag.re;
  v_im += ag.im;
  const C2<float> dv(v_re, v_im);
  const C2<float> ps = cdiv(dv, wn * C2<float>(-xi.re, -xi.im));
  ps_re = ps.re;
  ps_im = ps.im;
  rn = rn + cmul(dv, ps);
}

// x + alpha_prev p_prev + alpha p on two complex entries
__device__ __forceinline__ float4 add_two_terms(float4 x, float4 pp, float4 p, C2<float> alpha_prev, C2<float> alpha) {
  x.x += alpha_prev.re * pp.x - alpha_prev.im * pp.y;
  x.y += alpha_prev.re * pp.y + alpha_prev.im * pp.x;
  x.z += alpha_prev.re * pp.z - alpha_prev.im * pp.w;
  x.w += alpha_prev.re * pp.w + alpha_prev.im * pp.z;
  x.x += alpha.re * p.x - alpha.im * p.y;
  x.y += alpha.re * p.y + alpha.im * p.x;
  x.z += alpha.re * p.z - alpha.im * p.w;
  x.w += alpha.re * p.w + alpha.im * p.z;
  return x;
}

// Pairs in flight per thread in pass B: odd iterations read three more arrays
#ifndef TEM_UPD_U_ODD
#define TEM_UPD_U_ODD 2
#endif
#ifndef TEM_UPD_U_EVEN
#define TEM_UPD_U_EVEN 4
#endif

// Pointers and scalars of one slot's pass B on entry pairs.
struct UpdVec {
  C2<float> alpha, alpha_prev, xi;
  bool xzero;
  const float4 *a, *b, *ap, *bp, *q, *gp;
  float4 *w, *x, *xn, *u, *psi;
  const float2 *dK, *Me, *Wn;
};

// Edge pairs [from, to) with stride NT*U; ODD: also x += alpha_prev a_prev + alpha a.  Each
// thread has U pairs of every input in flight before it computes (U larger when the pass reads
// fewer arrays, so that about the same number of bytes are in flight).
template <bool ODD, int U>
__device__ __forceinline__ void update_edge_pairs(const UpdVec& P, int64_t from, int64_t to, C2<float>& rz, float& rr) {
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t base = from + threadIdx.x; base < to; base += (int64_t)NT * U) {
    float2 dk[U], me[U];
    float4 qr[U], wr[U], xr[U], ar[U], pr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = base + (int64_t)u * NT;
      if (p < to) {
        dk[u] = __ldg(P.dK + p);
        me[u] = __ldg(P.Me + p);
        qr[u] = __ldg(P.q + p);
        wr[u] = P.w[p];
        if (ODD) {
          ar[u] = __ldg(P.a + p);
          pr[u] = __ldg(P.ap + p);
          xr[u] = P.xzero ? z4 : P.x[p];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = base + (int64_t)u * NT;
      if (p >= to) continue;
      update_edge(wr[u].x, wr[u].y, qr[u].x, qr[u].y, dk[u].x, me[u].x, P.alpha, P.xi.re, P.xi.im, rz, rr);
      update_edge(wr[u].z, wr[u].w, qr[u].z, qr[u].w, dk[u].y, me[u].y, P.alpha, P.xi.re, P.xi.im, rz, rr);
      P.w[p] = wr[u];
      // boundary entries of both directions are 0, so x stays 0 there
      if (ODD) P.x[p] = add_two_terms(xr[u], pr[u], ar[u], P.alpha_prev, P.alpha);
    }
  }
}

// Node pairs [from, to) (indices within the nodal vectors); ODD: also x_n += alpha_prev b_prev + alpha b.
template <bool ODD, int U>
__device__ __forceinline__ void update_node_pairs(const UpdVec& P, int64_t from, int64_t to, C2<float>& rn) {
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t base = from + threadIdx.x; base < to; base += (int64_t)NT * U) {
    float2 wn[U];
    float4 gr[U], ur[U], xr[U], br[U], pr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t m = base + (int64_t)u * NT;
      if (m < to) {
        wn[u] = __ldg(P.Wn + m);
        gr[u] = __ldg(P.gp + m);
        ur[u] = P.u[m];
        if (ODD) {
          br[u] = __ldg(P.b + m);
          pr[u] = __ldg(P.bp + m);
          xr[u] = P.xzero ? z4 : P.xn[m];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t m = base + (int64_t)u * NT;
      if (m >= to) continue;
      float4 ps = z4;
      update_node(ur[u].x, ur[u].y, ps.x, ps.y, gr[u].x, gr[u].y, wn[u].x, P.alpha, P.xi, rn);
      update_node(ur[u].z, ur[u].w, ps.z, ps.w, gr[u].z, gr[u].w, wn[u].y, P.alpha, P.xi, rn);
      P.u[m] = ur[u];
      P.psi[m] = ps;
      if (ODD) P.xn[m] = add_two_terms(xr[u], pr[u], br[u], P.alpha_prev, P.alpha);
    }
  }
}

static __global__ void __launch_bounds__(NT, 3) k_cocg_update_vec(BatchArgs A) {
  __shared__ double red[NT / 32 * 4];
  const int2 bm = A.ublk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  if (!S->active) return;
  const SlotDesc& d = A.slots[slot];
  const int64_t nc = d.g.ncomp;
  UpdVec P;
  P.alpha = C2<float>(float(S->alpha_re), float(S->alpha_im));
  P.alpha_prev = C2<float>(float(S->alpha_prev_re), float(S->alpha_prev_im));
  P.xi = C2<float>(float(d.xi_re), float(d.xi_im));
  const bool odd = (S->iters & 1) != 0;             // this pass adds two terms to the correction
  P.xzero = S->iters == 1;                          // ... which starts at 0
  const int par = S->parity;                        // the direction written by pass A: a0/b0 if 1
  P.a = static_cast<const float4*>(par ? d.a0 : d.a1);
  P.b = static_cast<const float4*>(par ? d.b0 : d.b1);
  P.ap = static_cast<const float4*>(par ? d.a1 : d.a0);
  P.bp = static_cast<const float4*>(par ? d.b1 : d.b0);
  P.q = static_cast<const float4*>(d.q);
  P.gp = static_cast<const float4*>(d.gp);
  P.w = static_cast<float4*>(d.w);
  P.x = static_cast<float4*>(d.x);
  P.xn = static_cast<float4*>(d.xn);
  P.u = static_cast<float4*>(d.u);
  P.psi = static_cast<float4*>(d.psi);
  P.dK = reinterpret_cast<const float2*>(d.g.dKf);
  P.Me = reinterpret_cast<const float2*>(d.g.Mef);
  P.Wn = reinterpret_cast<const float2*>(d.g.Wnf);
  const int64_t ne2 = 3 * nc / 2, n2 = ne2 + (d.nodal ? nc / 2 : 0);
  const int64_t per = (n2 + d.nblk_update - 1) / d.nblk_update;
  const int64_t p0 = (int64_t)lb * per, p1 = min(n2, p0 + per);
  if (p1 > p0 && !TEM_CHECK(p1 - 1, n2, 12)) return;
  C2<float> rz = czero<float>(), rn = czero<float>();
  float rr = 0.f;
  const int64_t pe = min(p1, ne2), m0 = max(p0, ne2) - ne2, m1 = p1 - ne2;
  if (odd) {
    update_edge_pairs<true, TEM_UPD_U_ODD>(P, p0, pe, rz, rr);
    update_node_pairs<true, TEM_UPD_U_ODD>(P, m0, m1, rn);
  } else {
    update_edge_pairs<false, TEM_UPD_U_EVEN>(P, p0, pe, rz, rr);
    update_node_pairs<false, TEM_UPD_U_EVEN>(P, m0, m1, rn);
  }
  rz = rz + rn;
  double v[3] = {double(rz.re), double(rz.im), double(rr)};
  block_sum<3, NT>(v, red);
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<3>(v, part, A.ticket + slot, d.nblk_update, lb)) {
    double tot[3];
    sum_partials<3, NT>(part, d.nblk_update, tot, red);
    if (threadIdx.x != 0) return;
    finish_iteration(S, A.n_active, tot[0], tot[1], tot[2]);
  }
}

// ------------------------------ pass C: psi = D_n^{-1} G^T r;  rho = (r, D^-1 r) + (G^T r, psi)
// G^T r is not formed from r: in the air D_n is tiny, and rounding in the divergence of r
// would be amplified by 1/D_n.  Instead, with G^T K = 0 (curl grad = 0) and G^T b_outer = 0
// (the loop source and the adjoint sources are divergence-free), the residual of the inner
// solve A d = s r64 obeys exactly
//     G^T r_k = s xi G^T M x64 + xi G^T M d_k,    d_k = d_e + G d_n,
// so the first term (cn) is formed once, in FP64, when the solve starts.
template <class T>
__device__ __forceinline__ C2<T> nodal_at(const void* v, const GridView& g, int i, int j, int k, int64_t n) {
  // interior nodes only hold values; the boundary is zero
  if (i <= 0 || j <= 0 || k <= 0 || i >= g.nx || j >= g.ny || k >= g.nz) return czero<T>();
  return ld<T>(v, n);
}

// (G^T M v)_n at interior node n for an edge field v = v_e + G v_n (v_n may be NULL).
template <class T, class TV>
__device__ __forceinline__ C2<T> div_Mv(const Geo<T>& G, const GridView& g, const void* ve, const void* vn,
                                        int i, int j, int k, int64_t n) {
  const int64_t nc = g.ncomp, sy = g.nx, sz = (int64_t)g.nx * g.ny;
  auto edge_val = [&](int64_t e) {
    const C2<TV> v = ld<TV>(ve, e);
    return C2<T>(T(v.re), T(v.im));
  };
  auto node_val = [&](int ii, int jj, int kk, int64_t m) {
    if (!vn) return czero<T>();
    const C2<TV> v = nodal_at<TV>(vn, g, ii, jj, kk, m);
    return C2<T>(T(v.re), T(v.im));
  };
  const C2<T> v0 = node_val(i, j, k, n);
  // the six edges at n: x (i-1 -> i), x (i -> i+1), and likewise in y and z
  const C2<T> xm = edge_val(n - 1) + G.Rx[i - 1] * (v0 - node_val(i - 1, j, k, n - 1));
  const C2<T> xp = edge_val(n) + G.Rx[i] * (node_val(i + 1, j, k, n + 1) - v0);
  const C2<T> ym = edge_val(nc + n - sy) + G.Ry[j - 1] * (v0 - node_val(i, j - 1, k, n - sy));
  const C2<T> yp = edge_val(nc + n) + G.Ry[j] * (node_val(i, j + 1, k, n + sy) - v0);
  const C2<T> zm = edge_val(2 * nc + n - sz) + G.Rz[k - 1] * (v0 - node_val(i, j, k - 1, n - sz));
  const C2<T> zp = edge_val(2 * nc + n) + G.Rz[k] * (node_val(i, j, k + 1, n + sz) - v0);
  return (G.Rx[i - 1] * G.Me[n - 1]) * xm - (G.Rx[i] * G.Me[n]) * xp +
         (G.Ry[j - 1] * G.Me[nc + n - sy]) * ym - (G.Ry[j] * G.Me[nc + n]) * yp +
         (G.Rz[k - 1] * G.Me[2 * nc + n - sz]) * zm - (G.Rz[k] * G.Me[2 * nc + n]) * zp;
}

// (G^T v)_n at interior node n for an FP64 complex edge field v: +v / L on the three arriving
// edges, -v / L on the three leaving ones.
__device__ __forceinline__ C2<double> div_v(const Geo<double>& G, const GridView& g, const void* v, int i, int j,
                                            int k, int64_t n) {
  const int64_t nc = g.ncomp, sy = g.nx, sz = (int64_t)g.nx * g.ny;
  return G.Rx[i - 1] * ld<double>(v, n - 1) - G.Rx[i] * ld<double>(v, n) + G.Ry[j - 1] * ld<double>(v, nc + n - sy) -
         G.Ry[j] * ld<double>(v, nc + n) + G.Rz[k - 1] * ld<double>(v, 2 * nc + n - sz) -
         G.Rz[k] * ld<double>(v, 2 * nc + n);
}

// INIT: the pass that starts an armed solve (cn from x64 in FP64, d = 0); otherwise the
// pass that ends an iteration of an active solve.  For a right-hand side b with G^T b != 0
// (rhs_div) the start adds it: G^T r64 = G^T b + xi G^T M x64, so cn = s (G^T b + xi G^T M x64).
template <class T, bool INIT>
__global__ void __launch_bounds__(NT) k_cocg_nodal(BatchArgs A) {
  __shared__ double red[NT / 32 * 4];
  const int2 bm = A.nblk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  const bool pend = INIT;
  if (INIT ? !S->pending : !S->active) return;
  const SlotDesc& d = A.slots[slot];
  if (!d.nodal) return;
  const GridView& g = d.g;
  const Geo<T> G(g);
  const Geo<double> G64(g);
  const C2<T> xi(T(d.xi_re), T(d.xi_im));
  const C2<double> xi64(d.xi_re, d.xi_im);
  const double sc = 1.0 / S->inv_scale_prev;   // scale of this solve's right-hand side
  const void* x64 = d.x64[S->xcur];
  const uint32_t nn = (uint32_t)g.ncomp;
  const uint32_t per = (nn + d.nblk_nodal - 1) / d.nblk_nodal;
  const uint32_t n0 = (uint32_t)lb * per, n1 = min(nn, n0 + per);
  C2<T> rho = czero<T>();
  for (uint32_t n = n0 + threadIdx.x; n < n1; n += NT) {
    const uint32_t row = fdiv(n, d.div_nx);
    const int i = int(n - row * (uint32_t)g.nx);
    const uint32_t k = fdiv(row, d.div_ny);
    const int j = int(row - k * (uint32_t)g.ny);
    C2<T> ps = czero<T>();
    if (i > 0 && j > 0 && k > 0) {
      C2<T> dv;
      if (INIT) {  // start of a solve: cn = s xi G^T M x64 in FP64; d = 0
        C2<double> c0 = cmul(xi64, div_Mv<double, double>(G64, g, x64, nullptr, i, j, int(k), n));
        if (d.rhs_div) c0 = c0 + div_v(G64, g, d.rhs_c, i, j, int(k), n);
        c0 = sc * c0;
        dv = C2<T>(T(c0.re), T(c0.im));
        st<T>(d.cn, n, dv);
        st<T>(d.u, n, dv);   // v = cn + xi G^T M d with d = 0
      } else {
        dv = ld<T>(d.cn, n) + cmul(xi, div_Mv<T, T>(G, g, d.x, d.xn, i, j, int(k), n));
      }
      const C2<T> Dn = G.Wn[n] * C2<T>(-xi.re, -xi.im);
      ps = cdiv(dv, Dn);
      rho = rho + cmul(dv, ps);
    }
    st<T>(d.psi, n, ps);
  }
  double v[2] = {double(rho.re), double(rho.im)};
  block_sum<2, NT>(v, red);
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<2>(v, part, A.ticket + slot, d.nblk_nodal, lb)) {
    double tot[2];
    sum_partials<2, NT>(part, d.nblk_nodal, tot, red);
    if (threadIdx.x != 0) return;
    const double rre = S->rhoe_re + tot[0], rim = S->rhoe_im + tot[1];
    if (pend) {  // first nodal pass of an inner solve: rho_0 and the first beta
      S->pending = 0;
      start_direction(S, rre, rim);
      S->active = 1;
      return;
    }
    finish_iteration(S, A.n_active, rre, rim, S->rr);
  }
}

// ------------------------------- FP64 residual pass (the outer defect-correction step)
// x <- x64[cur] + inv_scale_prev (d_e + G d_n)  (the last inner correction), into x64[cur^1];
// r = b - A x in FP64;  w_inner = (scale r) / D  in the inner precision TI;
// then (last CTA) either finish the slot or arm the next inner COCG solve.
template <class TI>
struct ResidualPol {
  const void* xcur; const void* de; const void* dn; void* xnext; double inv_sc; bool upd;
  bool dok;                                   // de, dn hold the correction (else it starts at 0)
  const void* pe; const void* pn; C2<double> alag;   // the term the update passes left out (pe NULL: none)
  const double* f; const void* rhs_c;
  C2<double> xi; const double* Me;
  Geo<TI> GI; Geo<double> G; const GridView* g; TI xr, xim;
  void* win; double scale;
  double rr, rz_re, rz_im;
  __device__ ResidualPol(const GridView& gv) : GI(gv), G(gv), g(&gv) {}
  __device__ C2<double> load(int c, int i, int j, int k, int64_t idx, bool own) {
    C2<double> x = ld<double>(xcur, idx);
    if (upd && edge_valid(c, i, j, k)) {
      const int64_t n0 = i + (int64_t)g->nx * (j + (int64_t)g->ny * k);
      // d = d_e + G d_n, plus alag (p_e + G p_n) when the last update pass left that term out
      C2<double> corr = czero<double>();
      if (dok) corr = field_at(de, dn, c, i, j, k, idx, n0);
      if (pe) corr = corr + cmul(alag, field_at(pe, pn, c, i, j, k, idx, n0));
      x = x + inv_sc * corr;
      if (own) st<double>(xnext, idx, x);
    }
    return x;
  }
  // (v_e + G v_n) on edge (c, i, j, k) in double, from an edge and a nodal vector of type TI
  __device__ C2<double> field_at(const void* ve, const void* vn, int c, int i, int j, int k, int64_t idx,
                                 int64_t n0) const {
    const C2<TI> dv = ld<TI>(ve, idx);
    C2<double> f(double(dv.re), double(dv.im));
    if (vn) {
      const C2<TI> b0 = ld<TI>(vn, n0);
      const C2<TI> gb = grad_edge<TI>(GI, *g, c, i, j, k, n0, b0, vn, czero<TI>(), nullptr, nullptr, false);
      f = f + C2<double>(double(gb.re), double(gb.im));
    }
    return f;
  }
  template <class U> __device__ void node(int64_t, int, int, int, U, U, U) {}
  __device__ void prefetch(int64_t, int, int, int) {}
  template <class C, class U> __device__ void prev_plane(int64_t, int, int, int, C, U) {}
  template <class C, class U>
  __device__ void node_end(int64_t, int, int, int, C, C, C, U, U, U, U, U) {}
  __device__ void edge(int c, int64_t idx, int i, int j, int k, C2<double> xv, C2<double> kx) {
    const C2<double> ax = kx - cmul(xi, Me[idx] * xv);
    const C2<double> b = rhs_c ? ld<double>(rhs_c, idx) : C2<double>(f[idx], 0.0);
    const C2<double> r = b - ax;
    rr += r.re * r.re + r.im * r.im;
    const C2<TI> rs(TI(scale * r.re), TI(scale * r.im));
    const C2<TI> wv = cdiv(rs, jacobi_D<TI>(GI, c, i, j, k, idx, C2<TI>(xr, xim)));
    if (TEM_CHECK(idx, 3 * g->ncomp, 5)) st<TI>(win, idx, wv);
    const C2<TI> pz = cmul(rs, wv);
    rz_re += double(pz.re);
    rz_im += double(pz.im);
  }
  __device__ void edge_invalid(int64_t idx) {
    if (TEM_CHECK(idx, 3 * g->ncomp, 6)) st<TI>(win, idx, czero<TI>());
  }
};

template <class TI>
__global__ void __launch_bounds__(NT) k_residual(BatchArgs A, int* n_done) {
  __shared__ StencilSmem<double> sm;
  const int2 bm = A.blk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  if (S->done || S->active || S->pending) return;  // finished, or an inner solve is under way
  const SlotDesc d = A.slots[slot];
  int i0, j0, k0, k1;
  tile_of(d, lb, d.g.nz, i0, j0, k0, k1);
  ResidualPol<TI> pol(d.g);
  pol.upd = S->outer > 0;
  pol.xcur = d.x64[S->xcur];
  pol.xnext = d.x64[S->xcur ^ 1];
  pol.de = d.x;
  pol.dn = d.nodal ? d.xn : nullptr;
  // the update passes write the correction on odd iterations: it holds data once two
  // iterations are done, and lacks the last term when the solve ended after an even one
  pol.dok = S->iters >= 2;
  pol.pe = S->lag ? (S->lag_par ? d.a0 : d.a1) : nullptr;
  pol.pn = S->lag && d.nodal ? (S->lag_par ? d.b0 : d.b1) : nullptr;
  pol.alag = C2<double>(S->alpha_prev_re, S->alpha_prev_im);
  pol.inv_sc = S->inv_scale_prev;
  pol.f = d.f;
  pol.rhs_c = d.rhs_c;
  pol.xi = C2<double>(d.xi_re, d.xi_im);
  pol.Me = d.g.Me;
  pol.xr = TI(d.xi_re);
  pol.xim = TI(d.xi_im);
  pol.win = d.w;
  pol.scale = S->scale;
  pol.rr = pol.rz_re = pol.rz_im = 0.0;
  stencil_march<double>(sm, d.g, pol, i0, j0, k0, k1);
  double v[3] = {pol.rr, pol.rz_re, pol.rz_im};
  block_sum<3, NT>(v, sm.red);
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<3>(v, part, A.ticket + slot, d.nblk_stencil, lb)) {
    double tot[3];
    sum_partials<3, NT>(part, d.nblk_stencil, tot, sm.red);
    if (threadIdx.x != 0) return;
    if (pol.upd) S->xcur ^= 1;
    S->rr64 = tot[0];
    S->outer += 1;
    bool finish = false;
    if (!isfinite(tot[0])) {
      S->status = TEM_EBREAKDOWN;
      finish = true;
    } else if (tot[0] <= S->tol_outer2) {
      finish = true;
    } else if (S->status != TEM_OK) {
      finish = true;  // the last inner solve failed
    } else if (S->outer > S->max_outer || S->total_iters >= S->max_iter) {
      S->status = TEM_ENOCONV;
      finish = true;
    }
    if (finish) {
      S->done = 1;
      atomicAdd(n_done, 1);
      return;
    }
    // arm the inner solve on  A d = scale * r  (d = d_e + G d_n starts at 0)
    const double sc = S->scale;
    S->bb = sc * sc * tot[0];
    const double want = 0.25 * S->tol_outer2 / tot[0];   // reach 1/2 of the final target
    const double rel2 = d.fp64_inner ? want : fmax(S->inner_rel2, want);
    S->tol2 = rel2 * S->bb;
    S->iters = 0;
    S->lag = 0;
    S->rr_best = S->bb;
    S->it_best = 0;
    // continue the last inner solve's direction (residual replacement), or restart: first
    // outer step, carrying off, or the last inner solve stagnated
    const bool carry = S->carry && pol.upd && !S->stalled;
    S->stalled = 0;
    if (carry) {
      S->carry_ratio = sc * S->inv_scale_prev;  // s / s_prev (> 0)
      S->parity ^= 1;                           // the last direction becomes a_old, b_old
    } else {
      S->carry_ratio = 0.0;
      S->parity = 0;
    }
    S->inv_scale_prev = 1.0 / sc;
    S->scale = 1.0 / sqrt(tot[0]);
    S->rhoe_re = tot[1];
    S->rhoe_im = tot[2];
    if (d.nodal) {
      S->pending = 1;            // the nodal pass adds (G^T r, psi) to rho_0 and starts the solve
    } else {
      start_direction(S, tot[1], tot[2]);
      S->active = 1;
    }
    atomicAdd(A.n_active, 1);
  }
}

// ------------------------------------------------------ q = (K - xi M) p, s shifts
template <class T>
struct ApplyPol {
  const void* p; void* q; C2<T> xi; const T* Me;
  __device__ C2<T> load(int, int, int, int, int64_t idx, bool) { return ld<T>(p, idx); }
  __device__ void node(int64_t, int, int, int, T, T, T) {}
  __device__ void prefetch(int64_t, int, int, int) {}
  __device__ void prev_plane(int64_t, int, int, int, C2<T>, T) {}
  __device__ void node_end(int64_t, int, int, int, C2<T>, C2<T>, C2<T>, T, T, T, T, T) {}
  __device__ void edge(int, int64_t idx, int, int, int, C2<T> pv, C2<T> kp) {
    st<T>(q, idx, kp - cmul(xi, Me[idx] * pv));
  }
  __device__ void edge_invalid(int64_t idx) { st<T>(q, idx, czero<T>()); }
};

template <class T>
__global__ void __launch_bounds__(NT) k_apply(GridView g, const double* xi, const void* p, void* q,
                                              int tiles_x, int tiles_y, int zchunk) {
  __shared__ StencilSmem<T> sm;
  const int shift = blockIdx.y;
  const int lb = blockIdx.x;
  const int tx = lb % tiles_x, r = lb / tiles_x, ty = r % tiles_y, zc = r / tiles_y;
  const int i0 = tx * TX, j0 = ty * TY, k0 = zc * zchunk, k1 = min(k0 + zchunk, g.nz);
  const int64_t n = 3 * g.ncomp;
  typedef typename Vec2<T>::type V;
  ApplyPol<T> pol;
  pol.p = reinterpret_cast<const V*>(p) + shift * n;
  pol.q = reinterpret_cast<V*>(q) + shift * n;
  pol.xi = C2<T>(T(xi[2 * shift]), T(xi[2 * shift + 1]));
  pol.Me = Geo<T>(g).Me;
  stencil_march<T>(sm, g, pol, i0, j0, k0, k1);
}

// --------------------------------- receivers and the pole -> channel combination
// y[i][r] = sum_terms w x_i[edge];   d[r][k] = sum_i Re(c[i][k] y[i][r])   (Eq. (rmjQ))
static __global__ void k_project_combine(const SlotDesc* slots, const SlotScalars* sc, int s,
                                  const int64_t* term_edge, const double* term_w, const int* term_off,
                                  const double* c, int K, double* d, int n_rx) {
  __shared__ double ys[2 * 64];
  const int r = blockIdx.x;
  if (r >= n_rx) return;
  const int t0 = term_off[r], t1 = term_off[r + 1];
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const SlotDesc& dsc = slots[i];
    const void* x = dsc.x64[sc[i].xcur];
    double yr = 0.0, yi = 0.0;
    for (int t = t0; t < t1; ++t) {
      const C2<double> v = ld<double>(x, term_edge[t]);
      yr += term_w[t] * v.re;
      yi += term_w[t] * v.im;
    }
    ys[2 * i] = yr;
    ys[2 * i + 1] = yi;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < s; ++i) {
      const double cr = c[2 * (i * K + k)], ci = c[2 * (i * K + k) + 1];
      acc += cr * ys[2 * i] - ci * ys[2 * i + 1];
    }
    d[(int64_t)r * K + k] = acc;
  }
}

// y[i][r] alone (diagnostics and the cancellation factor)
static __global__ void k_project(const SlotDesc* slots, const SlotScalars* sc, int s,
                          const int64_t* term_edge, const double* term_w, const int* term_off,
                          double* y, int n_rx) {
  const int r = blockIdx.x;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const void* x = slots[i].x64[sc[i].xcur];
    double yr = 0.0, yi = 0.0;
    for (int t = term_off[r]; t < term_off[r + 1]; ++t) {
      const C2<double> v = ld<double>(x, term_edge[t]);
      yr += term_w[t] * v.re;
      yi += term_w[t] * v.im;
    }
    y[2 * ((int64_t)i * n_rx + r)] = yr;
    y[2 * ((int64_t)i * n_rx + r) + 1] = yi;
  }
}

// ------------------------------------------------------------- scatters
static __global__ void k_scatter(const int64_t* idx, const double* val, int64_t n, double* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[idx[t]] = val[t];
}
static __global__ void k_scatter_c(const int64_t* idx, const double* val, int64_t n, double* out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    out[2 * idx[t]] = val[2 * t];
    out[2 * idx[t] + 1] = val[2 * t + 1];
  }
}

// ------------------------------------------------------------- adjoint gradient
// g[cell] = sum_i Re( xi_i sigma_c V_c / 4 sum_{12 edges e of the cell} lam_i[e] x_i[e] )
static __global__ void k_gradient(GridView g, const double* sigma, const SlotDesc* fwd, const SlotScalars* fsc,
                           const SlotDesc* adj, const SlotScalars* asc, int s, double* grad) {
  const int64_t ncell = g.ncomp;
  for (int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cidx < ncell;
       cidx += (int64_t)gridDim.x * blockDim.x) {
    const int i = int(cidx % g.nx);
    const int64_t r = cidx / g.nx;
    const int j = int(r % g.ny), k = int(r / g.ny);
    const double q = 0.25 * sigma[cidx] * g.Lx[i] * g.Ly[j] * g.Lz[k];
    double acc = 0.0;
    for (int sh = 0; sh < s; ++sh) {
      const void* x = fwd[sh].x64[fsc[sh].xcur];
      const void* lam = adj[sh].x64[asc[sh].xcur];
      double sr = 0.0, si = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          int64_t e[3];
          bool ok[3];
          // x-edge (i, j+a, k+b), y-edge (i+a, j, k+b), z-edge (i+a, j+b, k)
          ok[0] = (j + a < g.ny) && (k + b < g.nz);
          e[0] = i + (int64_t)g.nx * ((j + a) + (int64_t)g.ny * (k + b));
          ok[1] = (i + a < g.nx) && (k + b < g.nz);
          e[1] = g.ncomp + (i + a) + (int64_t)g.nx * (j + (int64_t)g.ny * (k + b));
          ok[2] = (i + a < g.nx) && (j + b < g.ny);
          e[2] = 2 * g.ncomp + (i + a) + (int64_t)g.nx * ((j + b) + (int64_t)g.ny * k);
          for (int t = 0; t < 3; ++t) {
            if (!ok[t]) continue;
            const C2<double> xv = ld<double>(x, e[t]);
            const C2<double> lv = ld<double>(lam, e[t]);
            sr += lv.re * xv.re - lv.im * xv.im;
            si += lv.re * xv.im + lv.im * xv.re;
          }
        }
      const double xr = fwd[sh].xi_re, xim = fwd[sh].xi_im;
      acc += xr * sr - xim * si;
    }
    grad[cidx] = q * acc;
  }
}

// ------------------------------------------------- time snapshots of the field (Sec. 3.2)
// The columns of S R: u_k[e] = sum_i Re(c[i, k] x_i[e]) for k = k0 .. k0+nk-1, stored at
// out + (k - k0) * n3.  One thread per (edge, channel); the channel varies fastest over the
// blocks, so the nk blocks of one edge range run together and read the x_i of their range
// from L2 after the first of them brought it in: HBM sees x once and every output once.
static __global__ void __launch_bounds__(NT) k_fields(const SlotDesc* slots, const SlotScalars* sc, int s,
                                                      const double* c, int K, int k0, int nk, int64_t n3,
                                                      double* out) {
  __shared__ const double2* xp[64];
  __shared__ double2 cs[64];
  const int kk = int(blockIdx.x % (unsigned)nk);
  const int64_t e = (int64_t)(blockIdx.x / (unsigned)nk) * NT + threadIdx.x;
  for (int i = threadIdx.x; i < s; i += NT) {
    xp[i] = static_cast<const double2*>(slots[i].x64[sc[i].xcur]);
    cs[i] = make_double2(c[2 * (i * K + k0 + kk)], c[2 * (i * K + k0 + kk) + 1]);
  }
  __syncthreads();
  if (e >= n3) return;
  double acc = 0.0;
  for (int i = 0; i < s; ++i) {
    const double2 x = xp[i][e];
    acc += cs[i].x * x.x - cs[i].y * x.y;
  }
  __stcs(out + (int64_t)kk * n3 + e, acc);
}

// ------------------------------------------------- linearised forward (Sec. 4)
// b_i[e] = xi_i dM_e x_i[e] with dM_e = sum over the four cells around edge e of
// sigma_c dm_c V_c / 4 (the lumped mass with sigma replaced by sigma * dm); boundary and
// padding entries 0.  b_i is stored at rhs + i * 3 * ncomp (complex).
static __global__ void k_jvp_rhs(GridView g, const double* sigma, const double* dm, const SlotDesc* fwd,
                                 const SlotScalars* fsc, int s, double* rhs) {
  const int64_t nc = g.ncomp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = int(e / nc);
    const int64_t r = e - c * nc;
    const int i = int(r % g.nx);
    const int64_t r2 = r / g.nx;
    const int j = int(r2 % g.ny), k = int(r2 / g.ny);
    double m = 0.0;
    if (edge_valid(c, i, j, k)) {
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          int ci = i, cj = j, ck = k;
          if (c == 0) { cj = j - 1 + a; ck = k - 1 + b; }
          if (c == 1) { ci = i - 1 + a; ck = k - 1 + b; }
          if (c == 2) { ci = i - 1 + a; cj = j - 1 + b; }
          const int64_t cell = ci + (int64_t)g.nx * (cj + (int64_t)g.ny * ck);
          m += 0.25 * sigma[cell] * dm[cell] * g.Lx[ci] * g.Ly[cj] * g.Lz[ck];
        }
    }
    for (int sh = 0; sh < s; ++sh) {
      C2<double> b = czero<double>();
      if (m != 0.0) {
        const C2<double> xv = ld<double>(fwd[sh].x64[fsc[sh].xcur], e);
        b = cmul(C2<double>(fwd[sh].xi_re * m, fwd[sh].xi_im * m), xv);
      }
      st<double>(rhs + (int64_t)sh * 6 * nc, e, b);
    }
  }
}

// Per-slot ||b_i||^2 partials: block (b, i) sums |b_i|^2 over its fixed chunk into
// part[i * gridDim.x + b]; the host adds the partials in order.
static __global__ void k_rhs_norm2(const double* rhs, int64_t n, double* part) {
  __shared__ double red[NT / 32];
  const int sh = blockIdx.y;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = (int64_t)blockIdx.x * per, e1 = e0 + per < n ? e0 + per : n;
  const double* v = rhs + (int64_t)sh * 2 * n;
  double acc[1] = {0.0};
  for (int64_t e = e0 + threadIdx.x; e < e1; e += NT) acc[0] += v[2 * e] * v[2 * e] + v[2 * e + 1] * v[2 * e + 1];
  block_sum<1, NT>(acc, red);
  if (threadIdx.x == 0) part[(int64_t)sh * gridDim.x + blockIdx.x] = acc[0];
}

}  // namespace tem

#include "stencil_tma.cuh"
