// Pass A of the FP32 COCG sweeps with tile loads by the tensor memory accelerator (TMA).
//
// The same arithmetic as k_cocg_stencil_pipe (kernels.cuh): for every own node (i, j, k) of a
// 32 x 8 column of nodes marched over a z chunk,
//   a = w + beta a_old,  b = psi + beta b_old        (the new search direction, p = a + G b),
//   q = (K - xi M) a - xi M G b                      (Sec. 2.2: K from the Yee face circulations),
//   (p, q) partial sums,  G^T M p at interior nodes  (the nodal part of the preconditioner).
//
// Data movement.  One elected thread issues, per z plane, one TMA box per input array into a ring
// of shared-memory stages, completing on an mbarrier per stage:
//   w (3 components) and psi, boxed as 36 x 10 complex (x from i0-2: a 16-byte aligned start),
//   a_old (3 components) and b_old (only when beta != 0),
//   the packed FP32 masses (M_x, M_y, M_z, W_n) per node, 34 x 9 records.
// Positions outside the grid arrive as zeros (out-of-bounds fill), which is the value every
// vector holds there.  a and b are formed in place in the landed stage; each thread then
// computes the faces its three edges need straight from the formed planes (its own faces and
// those at i-1 and j-1; the faces one plane below stay in registers).  Two CTA barriers per
// plane: one frees the stage that the next TMA load overwrites, the other separates forming
// plane k+1 from reading it.
//
// Planes k0-1 .. k1 pass through the ring; plane p uses W/M stage (p - k0 + 1) mod NW and
// a_old stage (p - k0 + 1) mod NO.  Each step k starts with a barrier (everyone is done with
// plane k-1), issues plane k+2 into plane k-1's stage, then waits for plane k+1 and forms it:
// two planes are in flight while a third is formed and computed.
//
// Every wait on an mbarrier is bounded (about one second of device time).  A CTA whose wait
// runs out marks its slot TEM_ETIMEOUT and inactive, waits (again bounded) for the loads it
// issued and still publishes its partial sums, so that the slot's ticket stays consistent.
#pragma once

#include <cuda.h>

namespace tem {
namespace tma {

constexpr int BX = TX + 4;        // 36 complex columns: i0-2 .. i0+33
constexpr int BY = TY + 2;        // 10 rows: j0-1 .. j0+8
constexpr int PL = BX * BY;       // complex entries of one component plane
constexpr int MX = TX + 2;        // 34 mass columns: i0-2 .. i0+31
constexpr int MY = TY + 1;        // 9 mass rows: j0-1 .. j0+7
#ifndef TEM_TMA_NW
#define TEM_TMA_NW 3              // formed / landing planes (k, k+1, k+2)
#endif
constexpr int NW = TEM_TMA_NW;
constexpr int NO = 2;             // raw a_old / b_old planes
static_assert(NW >= 3, "planes k, k+1 and k+2 need their own stages");

// byte layout of one stage (TMA destinations 128-byte aligned)
constexpr unsigned VEC_B = 3u * PL * 8u;                  // 3 components, dense (one box)
constexpr unsigned NOD_OFF = (VEC_B + 127u) & ~127u;      // nodal plane after the components
constexpr unsigned NOD_B = PL * 8u;
constexpr unsigned STAGE_B = (NOD_OFF + NOD_B + 127u) & ~127u;
constexpr unsigned MASS_B = MY * MX * 16u;
constexpr unsigned MSTAGE_B = (MASS_B + 127u) & ~127u;
constexpr unsigned W_OFF = 0;
constexpr unsigned O_OFF = W_OFF + NW * STAGE_B;
constexpr unsigned M_OFF = O_OFF + NO * STAGE_B;
constexpr unsigned RED_OFF = M_OFF + NW * MSTAGE_B;
constexpr unsigned BAR_OFF = RED_OFF + (NT / 32) * 4 * 8;
constexpr unsigned FLAG_OFF = BAR_OFF + NW * 8;
constexpr int ZG = ZMAX + 2;                              // z geometry of planes k0-1 .. k1
constexpr unsigned ZG_OFF = FLAG_OFF + 16;
constexpr unsigned SMEM_B = ZG_OFF + 3 * ZG * 4 + 128;    // + slack to align the base to 128

// tensor maps of one slot, in this order
enum { MAP_W = 0, MAP_A0, MAP_A1, MAP_PSI, MAP_B0, MAP_B1, MAP_MQ, NMAP };

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// One bounded try: the warp sleeps until the phase completes or about 0.1 ms pass.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for phase `parity` of barrier b; false after about one second.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(b, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}
__device__ __forceinline__ void load3(void* dst, const CUtensorMap* m, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::
          "r"(su32(dst)), "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void load4(void* dst, const CUtensorMap* m, int c0, int c1, int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::
          "r"(su32(dst)), "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(bar))
      : "memory");
}

struct Ring {
  unsigned char* base;
  __device__ float2* vec(int s) const { return reinterpret_cast<float2*>(base + W_OFF + s * STAGE_B); }
  __device__ float2* nod(int s) const { return reinterpret_cast<float2*>(base + W_OFF + s * STAGE_B + NOD_OFF); }
  __device__ float2* ovec(int s) const { return reinterpret_cast<float2*>(base + O_OFF + s * STAGE_B); }
  __device__ float2* onod(int s) const { return reinterpret_cast<float2*>(base + O_OFF + s * STAGE_B + NOD_OFF); }
  __device__ float4* mass(int s) const { return reinterpret_cast<float4*>(base + M_OFF + s * MSTAGE_B); }
  __device__ double* red() const { return reinterpret_cast<double*>(base + RED_OFF); }
  __device__ uint64_t* bar(int s) const { return reinterpret_cast<uint64_t*>(base + BAR_OFF) + s; }
  __device__ int* flag() const { return reinterpret_cast<int*>(base + FLAG_OFF); }
  __device__ float* zg() const { return reinterpret_cast<float*>(base + ZG_OFF); }   // [3][ZG]: Lz, 1/Lz, Sz/mu0
};

// Issue the loads of plane p (one thread): W/M stage sw, a_old stage so, completion on bar(sw).
__device__ __forceinline__ void issue_plane(const Ring& R, const CUtensorMap* maps, int p, int sw, int so, int i0,
                                            int j0, bool nodal, bool use_beta, int aold, int bold) {
  uint64_t* bar = R.bar(sw);
  unsigned bytes = VEC_B + MASS_B + (nodal ? NOD_B : 0u);
  if (use_beta) bytes += VEC_B + (nodal ? NOD_B : 0u);
  mbar_expect_tx(bar, bytes);
  const int x0 = 2 * (i0 - 2);   // float coordinate of column i0-2 (a multiple of 4: 16 bytes)
  if (!TEM_CHECK(x0 & 3, 1, 7)) return;   // a misaligned box start: record it, issue nothing
  load4(R.vec(sw), maps + MAP_W, x0, j0 - 1, p, 0, bar);
  if (nodal) load3(R.nod(sw), maps + MAP_PSI, x0, j0 - 1, p, bar);
  load4(R.mass(sw), maps + MAP_MQ, 0, i0 - 2, j0 - 1, p, bar);
  if (use_beta) {
    load4(R.ovec(so), maps + aold, x0, j0 - 1, p, 0, bar);
    if (nodal) load3(R.onod(so), maps + bold, x0, j0 - 1, p, bar);
  }
}

// The pair of box entries a thread forms (threads 0 .. PL/2-1 each own one pair, in every array):
// its index among the 180 pairs of a component plane and, if the pair is an own entry of the
// tile inside the grid, its float4 index within a z plane of the global vectors (else -1).
struct FormPos {
  int m;          // pair index, or -1 for threads without a pair
  int g;          // (i + nx j) / 2 of the pair's first entry, or -1
};

__device__ __forceinline__ FormPos form_pos(int i0, int j0, int nx, int ny) {
  FormPos f;
  f.m = -1;
  f.g = -1;
  const int t = threadIdx.x;
  if (t >= PL / 2) return f;
  f.m = t;
  const int r = t / (BX / 2), pc = t - r * (BX / 2);
  const int i = i0 - 2 + 2 * pc, j = j0 - 1 + r;
  if (r >= 1 && r <= TY && pc >= 1 && pc <= TX / 2 && i < nx && j < ny) f.g = (i + nx * j) >> 1;   // nx even
  return f;
}

// Form plane p in place: a = w + beta a_old (3 components), b = psi + beta b_old, two complex
// entries per 16-byte access; own entries go to anew / bnew when the plane is an own plane
// (plane4 = first float4 of plane p, nc4 = float4 entries per component).
__device__ __forceinline__ void form_plane(const Ring& R, int sw, int so, const FormPos& f, int64_t plane4,
                                           bool store, int64_t nc4, bool nodal, bool use_beta, float br, float bi,
                                           float4* __restrict__ anew, float4* __restrict__ bnew) {
  if (f.m < 0) return;
  constexpr int HALF = PL / 2;
  float4* W = reinterpret_cast<float4*>(R.vec(sw)) + f.m;
  const float4* O = reinterpret_cast<const float4*>(R.ovec(so)) + f.m;
  const bool st = store && f.g >= 0;
  float4* ga = anew + plane4 + f.g;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (c == 3) {
      if (!nodal) break;
      W = reinterpret_cast<float4*>(R.nod(sw)) + f.m;
      O = reinterpret_cast<const float4*>(R.onod(so)) + f.m;
      ga = bnew + plane4 + f.g;
    }
    const int off = c < 3 ? c * HALF : 0;
    float4 v = W[off];
    if (use_beta) {
      const float4 o = O[off];
      v.x += br * o.x - bi * o.y;
      v.y += br * o.y + bi * o.x;
      v.z += br * o.z - bi * o.w;
      v.w += br * o.w + bi * o.z;
      W[off] = v;
    }
    if (st && TEM_CHECK(plane4 + f.g + (c < 3 ? c * nc4 : 0), c < 3 ? 3 * nc4 : nc4, 8)) ga[c < 3 ? c * nc4 : 0] = v;
  }
}

}  // namespace tma

// Rows of the box are 16-byte aligned only for an even nx; the tensor maps need that.
__host__ __device__ inline bool tma_layout_ok(const GridView& g) { return (g.nx % 2) == 0; }

template <bool NODAL>
__global__ void __launch_bounds__(NT, 3) k_cocg_stencil_tma(BatchArgs A) {
  using namespace tma;
  extern __shared__ unsigned char smem_raw[];
  Ring R;
  R.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int2 bm = A.blk2slot[blockIdx.x];
  const int slot = bm.x, lb = bm.y;
  SlotScalars* S = A.sc + slot;
  if (!S->active) return;
  const SlotDesc& d = A.slots[slot];
  // the grid's sizes and pointers in registers (the descriptor lives in global memory)
  const int nx = d.g.nx, ny = d.g.ny, nz = d.g.nz;
  const int64_t nc = d.g.ncomp, sxy = (int64_t)nx * ny;
  int i0, j0, k0, k1;
  tile_of(d, lb, nz, i0, j0, k0, k1);
  const CUtensorMap* maps = A.tmaps + (int64_t)slot * NMAP;
  const bool use_beta = !(S->beta_re == 0.0 && S->beta_im == 0.0);
  constexpr bool nodal = NODAL;   // the same for every slot of a launch
  const int par = S->parity;
  const int aold = par ? MAP_A1 : MAP_A0, bold = par ? MAP_B1 : MAP_B0;
  float4* anew = static_cast<float4*>(par ? d.a0 : d.a1);
  float4* bnew = static_cast<float4*>(par ? d.b0 : d.b1);
  float2* __restrict__ q = static_cast<float2*>(d.q);
  float2* __restrict__ gpo = static_cast<float2*>(d.gp);
  const float br = use_beta ? float(S->beta_re) : 0.f, bi = use_beta ? float(S->beta_im) : 0.f;
  const float xr = float(d.xi_re), xim = float(d.xi_im);
  const float* __restrict__ Lzf = d.g.Lzf;
  const float* __restrict__ Rzf = d.g.Rzf;
  const float* __restrict__ Szf = d.g.Szf;
  const bool leader = threadIdx.x == 0;
  const float inv_mu0 = float(1.0 / TEM_MU0);

  if (leader) {
    for (int s = 0; s < NW; ++s) mbar_init(R.bar(s), 1);
    *R.flag() = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (leader) {
    issue_plane(R, maps, k0 - 1, 0, 0, i0, j0, nodal, use_beta, aold, bold);
    issue_plane(R, maps, k0, 1, 1, i0, j0, nodal, use_beta, aold, bold);
  }
  // z geometry of planes k0-1 .. k1 (zero outside the grid), per-thread x/y geometry
  float* zg = R.zg();
  for (int t = threadIdx.x; t <= k1 - k0 + 1; t += NT) {
    const int k = k0 - 1 + t;
    const bool in = k >= 0 && k < nz;
    zg[t] = in ? Lzf[k] : 0.f;
    zg[ZG + t] = in ? Rzf[k] : 0.f;
    zg[2 * ZG + t] = in ? Szf[k] * inv_mu0 : 0.f;
  }
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = i0 + tx, j = j0 + ty;
  const bool mine = i < nx && j < ny;
  const float Lx = mine ? d.g.Lxf[i] : 0.f, Rx = mine ? d.g.Rxf[i] : 0.f, sx = mine ? d.g.Sxf[i] * inv_mu0 : 0.f;
  const float Ly = mine ? d.g.Lyf[j] : 0.f, Ry = mine ? d.g.Ryf[j] : 0.f, sy = mine ? d.g.Syf[j] * inv_mu0 : 0.f;
  const float Rxm = (mine && i > 0) ? d.g.Rxf[i - 1] : 0.f, Rym = (mine && j > 0) ? d.g.Ryf[j - 1] : 0.f;
  const int o = (ty + 1) * BX + (tx + 2);       // own entry in a component plane
  const int mo = (ty + 1) * MX + (tx + 2);      // own mass record
  const FormPos fp = form_pos(i0, j0, nx, ny);
  const int64_t nc4 = nc >> 1, sxy4 = sxy >> 1;  // float4 strides (nc, sxy even)
  // planes are counted from k0-1: plane k0-1+u uses W/M stage u mod NW and completes phase u / NW
  int issued = 2, waited = 0;                    // loads issued / seen complete (leader's count)
  bool ok = mbar_wait(R.bar(0), 0);
  if (ok) {
    waited = 1;
    form_plane(R, 0, 0, fp, sxy4 * (k0 - 1), false, nc4, nodal, use_beta, br, bi, anew, bnew);
  } else {
    *R.flag() = 1;
  }
  __syncthreads();   // plane k0-1 is formed: its a_old stage takes plane k0+1 while plane k0 lands
  bool abort = *R.flag() != 0;
  if (!abort && k0 + 1 <= k1) {
    if (leader) {
      fence_proxy_async();
      issue_plane(R, maps, k0 + 1, 2, 0, i0, j0, nodal, use_beta, aold, bold);
    }
    issued = 3;
  }
  if (!abort) {
    ok = mbar_wait(R.bar(1), 0);
    if (ok) {
      waited = 2;
      form_plane(R, 1, 1, fp, sxy4 * k0, true, nc4, nodal, use_beta, br, bi, anew, bnew);
    } else {
      *R.flag() = 1;
    }
  }
  __syncthreads();
  abort = *R.flag() != 0;
  // the column one plane below the chunk: F_x, F_y there, a_z, b, M_z and 1/Lz
  float2 fxm = make_float2(0.f, 0.f), fym = fxm, az_prev = fxm, b_prev = fxm;
  float mz_prev = 0.f, rz_prev = 0.f;
  if (mine && !abort) {
    const float2* P0 = R.vec(0);
    const float2* P1 = R.vec(1);
    az_prev = P0[2 * PL + o];
    b_prev = nodal ? R.nod(0)[o] : make_float2(0.f, 0.f);
    if (k0 > 0) {
      const float rz = zg[ZG];
      const float2 py = P0[PL + o], pyk = P1[PL + o], pz = P0[2 * PL + o], pzj = P0[2 * PL + o + BX];
      const float2 px = P0[o], pxk = P1[o], pzi = P0[2 * PL + o + 1];
      fxm.x = sx * (rz * (py.x - pyk.x) + Ry * (pzj.x - pz.x));
      fxm.y = sx * (rz * (py.y - pyk.y) + Ry * (pzj.y - pz.y));
      fym.x = sy * (Rx * (pz.x - pzi.x) + rz * (pxk.x - px.x));
      fym.y = sy * (Rx * (pz.y - pzi.y) + rz * (pxk.y - px.y));
      mz_prev = R.mass(0)[mo].z;
      rz_prev = rz;
    }
  }
  float accr = 0.f, acci = 0.f;
  // own entries of plane k: q + n, gp + n with n = i + nx j + sxy k
  float2* qk = q + (i + (int64_t)nx * j) + sxy * k0;
  float2* gk = gpo + (i + (int64_t)nx * j) + sxy * k0;
#pragma unroll 1
  for (int k = k0; k < k1 && !abort; ++k, qk += sxy, gk += sxy) {
    const int sk = (k - k0 + 1) % NW, sk1 = (k - k0 + 2) % NW;
    // plane k+2 into the stage of plane k-1 before waiting for plane k+1, so that two planes are
    // in flight: the barrier says that everyone has passed the last use of that stage (the
    // arithmetic of plane k-1, or the column below at the chunk start).  Its a_old stage held
    // plane k, formed before the previous barrier.
    __syncthreads();
    if (k + 2 <= k1) {
      if (leader) {
        fence_proxy_async();
        issue_plane(R, maps, k + 2, (k + 3 - k0) % NW, (k + 3 - k0) % NO, i0, j0, nodal, use_beta, aold, bold);
      }
      issued = k - k0 + 4;
    }
    // plane k+1 (count k-k0+2): landed -> formed
    ok = mbar_wait(R.bar(sk1), (unsigned)(((k - k0 + 2) / NW) & 1));
    if (ok) {
      waited = k - k0 + 3;
      form_plane(R, sk1, (k - k0 + 2) % NO, fp, sxy4 * (k + 1), k + 1 < k1, nc4, nodal, use_beta, br, bi, anew, bnew);
    } else {
      *R.flag() = 1;
    }
    __syncthreads();
    abort = *R.flag() != 0;
    if (abort) break;
    if (!mine) continue;
    const float2* P = R.vec(sk);
    const float2* P1 = R.vec(sk1);
    const float4* Mk = R.mass(sk);
    const int zk = k - k0 + 1;
    const float lz = zg[zk], rz = zg[ZG + zk], sz = zg[2 * ZG + zk];
    // formed a on plane k around the own node and on plane k+1
    const float2 ax = P[o], ay = P[PL + o], az = P[2 * PL + o];
    const float2 ax_i = P[o - 1], ay_i = P[PL + o - 1], az_i = P[2 * PL + o - 1];
    const float2 ax_j = P[o - BX], ay_j = P[PL + o - BX], az_j = P[2 * PL + o - BX];
    const float2 ay_ip = P[PL + o + 1], az_ip = P[2 * PL + o + 1];
    const float2 ax_jp = P[o + BX], az_jp = P[2 * PL + o + BX];
    const float2 ax_ijp = P[o - 1 + BX], ay_ipjm = P[PL + o + 1 - BX];
    const float2 ax1 = P1[o], ay1 = P1[PL + o], ax1_i = P1[o - 1], ay1_j = P1[PL + o - BX];
    // faces: own F_x, F_y, F_z; F_y, F_z at i-1; F_x, F_z at j-1
    float2 fx, fy, fz, fyi, fzi, fxj, fzj;
    fx.x = sx * (rz * (ay.x - ay1.x) + Ry * (az_jp.x - az.x));
    fx.y = sx * (rz * (ay.y - ay1.y) + Ry * (az_jp.y - az.y));
    fy.x = sy * (Rx * (az.x - az_ip.x) + rz * (ax1.x - ax.x));
    fy.y = sy * (Rx * (az.y - az_ip.y) + rz * (ax1.y - ax.y));
    fz.x = sz * (Ry * (ax.x - ax_jp.x) + Rx * (ay_ip.x - ay.x));
    fz.y = sz * (Ry * (ax.y - ax_jp.y) + Rx * (ay_ip.y - ay.y));
    fyi.x = sy * (Rxm * (az_i.x - az.x) + rz * (ax1_i.x - ax_i.x));
    fyi.y = sy * (Rxm * (az_i.y - az.y) + rz * (ax1_i.y - ax_i.y));
    fzi.x = sz * (Ry * (ax_i.x - ax_ijp.x) + Rxm * (ay.x - ay_i.x));
    fzi.y = sz * (Ry * (ax_i.y - ax_ijp.y) + Rxm * (ay.y - ay_i.y));
    fxj.x = sx * (rz * (ay_j.x - ay1_j.x) + Rym * (az.x - az_j.x));
    fxj.y = sx * (rz * (ay_j.y - ay1_j.y) + Rym * (az.y - az_j.y));
    fzj.x = sz * (Rym * (ax_j.x - ax.x) + Rx * (ay_ipjm.x - ay_j.x));
    fzj.y = sz * (Rym * (ax_j.y - ax.y) + Rx * (ay_ipjm.y - ay_j.y));
    float2 kp[3];
    kp[0] = make_float2(Lx * ((fz.x - fzj.x) - (fy.x - fym.x)), Lx * ((fz.y - fzj.y) - (fy.y - fym.y)));
    kp[1] = make_float2(Ly * ((fx.x - fxm.x) - (fz.x - fzi.x)), Ly * ((fx.y - fxm.y) - (fz.y - fzi.y)));
    kp[2] = make_float2(lz * ((fy.x - fyi.x) - (fx.x - fxj.x)), lz * ((fy.y - fyi.y) - (fx.y - fxj.y)));
    // p = a + G b on the three leaving edges
    float2 pc[3] = {ax, ay, az};
    float2 b0 = make_float2(0.f, 0.f);
    if (nodal) {
      const float2* B = R.nod(sk);
      b0 = B[o];
      const float2 bxp = B[o + 1], byp = B[o + BX], bzp = R.nod(sk1)[o];
      pc[0].x += Rx * (bxp.x - b0.x); pc[0].y += Rx * (bxp.y - b0.y);
      pc[1].x += Ry * (byp.x - b0.x); pc[1].y += Ry * (byp.y - b0.y);
      pc[2].x += rz * (bzp.x - b0.x); pc[2].y += rz * (bzp.y - b0.y);
    }
    const float4 mq = Mk[mo];
    const float mc[3] = {mq.x, mq.y, mq.z};
    const bool valid[3] = {j > 0 && k > 0, i > 0 && k > 0, i > 0 && j > 0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 qv = make_float2(0.f, 0.f);
      if (valid[c]) {
        const float mr = mc[c] * pc[c].x, mi = mc[c] * pc[c].y;
        qv.x = kp[c].x - (xr * mr - xim * mi);
        qv.y = kp[c].y - (xr * mi + xim * mr);
        accr += pc[c].x * qv.x - pc[c].y * qv.y;
        acci += pc[c].x * qv.y + pc[c].y * qv.x;
      }
      if (TEM_CHECK(i + (int64_t)nx * j + sxy * k + c * nc, 3 * nc, 9)) qk[c * nc] = qv;
    }
    if (nodal && i > 0 && j > 0 && k > 0) {
      // (G^T M p)_n: +M p / L on the three arriving edges, -M p / L on the three leaving ones
      const float2* B = R.nod(sk);
      const float2 bxm = B[o - 1], bym = B[o - BX];
      const float mxm = Mk[mo - 1].x, mym = Mk[mo - MX].y;
      const float2 pxm = make_float2(ax_i.x + Rxm * (b0.x - bxm.x), ax_i.y + Rxm * (b0.y - bxm.y));
      const float2 pym = make_float2(ay_j.x + Rym * (b0.x - bym.x), ay_j.y + Rym * (b0.y - bym.y));
      const float2 pzm = make_float2(az_prev.x + rz_prev * (b0.x - b_prev.x), az_prev.y + rz_prev * (b0.y - b_prev.y));
      const float cx = Rxm * mxm, cy = Rym * mym, cz = rz_prev * mz_prev;
      const float ox = Rx * mq.x, oy = Ry * mq.y, oz = rz * mq.z;
      float2 v;
      v.x = cx * pxm.x + cy * pym.x + cz * pzm.x - ox * pc[0].x - oy * pc[1].x - oz * pc[2].x;
      v.y = cx * pxm.y + cy * pym.y + cz * pzm.y - ox * pc[0].y - oy * pc[1].y - oz * pc[2].y;
      if (TEM_CHECK(i + (int64_t)nx * j + sxy * k, nc, 10)) *gk = v;
    }
    fxm = fx;
    fym = fy;
    az_prev = az;
    b_prev = b0;
    mz_prev = mq.z;
    rz_prev = rz;
  }
  if (abort) {
    // drain: wait (bounded) for every plane this CTA issued, then leave the slot marked
    if (leader) {
      for (int p = waited; p < issued; ++p) mbar_wait(R.bar(p % NW), (unsigned)((p / NW) & 1));
      S->status = TEM_ETIMEOUT;
      if (atomicCAS(&S->active, 1, 0) == 1) atomicSub(A.n_active, 1);
    }
  }
  double v[2] = {double(accr), double(acci)};
  block_sum<2, NT>(v, R.red());
  double* part = A.part + (int64_t)slot * A.part_stride;
  if (publish_partial<2>(v, part, A.ticket + slot, d.nblk_stencil, lb)) {
    double tot[2];
    sum_partials<2, NT>(part, d.nblk_stencil, tot, R.red());
    if (threadIdx.x != 0) return;
    if (S->status == TEM_ETIMEOUT) return;
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

// Launch pass A through the TMA kernel (dynamic shared memory above 48 KB); nodal: the
// preconditioner of every slot in the launch has the nodal part.
static inline cudaError_t launch_stencil_tma(const BatchArgs& A, int nblk, bool nodal, cudaStream_t st) {
  static bool attr_done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_cocg_stencil_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tma::SMEM_B);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_cocg_stencil_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)tma::SMEM_B);
    if (e != cudaSuccess) return e;
    attr_done[dev] = true;
  }
  if (nodal)
    k_cocg_stencil_tma<true><<<nblk, NT, tma::SMEM_B, st>>>(A);
  else
    k_cocg_stencil_tma<false><<<nblk, NT, tma::SMEM_B, st>>>(A);
  return cudaGetLastError();
}

// Resident CTAs per SM of the TMA stencil (0 on error).
static inline int stencil_tma_occupancy() {
  int n = 0;
  if (cudaFuncSetAttribute(k_cocg_stencil_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tma::SMEM_B) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cocg_stencil_tma<true>, NT, tma::SMEM_B) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace tem
