// Host-side geometry: the loop source f and the receiver rows q_r as sparse
// term lists in the device edge layout.
//
// Source (Sec. 2.1, the step-off transmitter q; Sec. 2.2, [f]_i = (q, Phi_i)):
// a line current I along an edge of length L gives f_e = I L (+-1, the sign of
// the traversal).  Receiver (Sec. 5, the observation operator Q): d_t b_z =
// -(curl e)_z, with (curl e)_z on a z-face = circulation / area, interpolated
// bilinearly between the face centres of the node plane nearest the receiver.
#include <cmath>
#include <map>

#include "tem_internal.h"

namespace tem {

static bool edge_valid_host(int c, int i, int j, int k, int nx, int ny, int nz) {
  if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return false;
  return c == 0 ? (j > 0 && k > 0) : (c == 1 ? (i > 0 && k > 0) : (i > 0 && j > 0));
}

static int64_t edge_index(int c, int i, int j, int k, int nx, int ny, int nz) {
  return (int64_t)c * nx * ny * nz + i + (int64_t)nx * (j + (int64_t)ny * k);
}

int build_source(const tem_grid* g, const double* loop_xy, int64_t nv, double z_loop, double current,
                 std::vector<Term>& f) {
  f.clear();
  if (!loop_xy || nv < 3 || nv > 100000 || !std::isfinite(current)) return TEM_EINVAL;
  const int nx = g->v.nx, ny = g->v.ny, nz = g->v.nz;
  int k;
  if (locate_node(g->hz, g->origin[2], z_loop, &k) != TEM_OK) return TEM_EINVAL;
  std::vector<int> I(nv), J(nv);
  for (int64_t v = 0; v < nv; ++v) {
    if (!std::isfinite(loop_xy[2 * v]) || !std::isfinite(loop_xy[2 * v + 1])) return TEM_EINVAL;
    if (locate_node(g->hx, g->origin[0], loop_xy[2 * v], &I[v]) != TEM_OK) return TEM_EINVAL;
    if (locate_node(g->hy, g->origin[1], loop_xy[2 * v + 1], &J[v]) != TEM_OK) return TEM_EINVAL;
  }
  std::map<int64_t, double> acc;
  for (int64_t v = 0; v < nv; ++v) {
    const int ia = I[v], ja = J[v], ib = I[(v + 1) % nv], jb = J[(v + 1) % nv];
    if (ia != ib && ja != jb) return TEM_EINVAL;  // segments must follow grid lines
    if (ja == jb) {
      const double sgn = ib > ia ? 1.0 : -1.0;
      for (int i = std::min(ia, ib); i < std::max(ia, ib); ++i)
        if (edge_valid_host(0, i, ja, k, nx, ny, nz))
          acc[edge_index(0, i, ja, k, nx, ny, nz)] += current * g->hx[i] * sgn;
    } else {
      const double sgn = jb > ja ? 1.0 : -1.0;
      for (int j = std::min(ja, jb); j < std::max(ja, jb); ++j)
        if (edge_valid_host(1, ia, j, k, nx, ny, nz))
          acc[edge_index(1, ia, j, k, nx, ny, nz)] += current * g->hy[j] * sgn;
    }
  }
  for (auto& kv : acc)
    if (kv.second != 0.0) f.push_back(Term{kv.first, kv.second});
  return f.empty() ? TEM_EINVAL : TEM_OK;
}

int build_receiver(const tem_grid* g, const double* xyz, std::vector<Term>& q) {
  q.clear();
  const int nx = g->v.nx, ny = g->v.ny, nz = g->v.nz;
  double ext[3] = {0, 0, 0};
  for (double w : g->hx) ext[0] += w;
  for (double w : g->hy) ext[1] += w;
  for (double w : g->hz) ext[2] += w;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(xyz[a])) return TEM_EINVAL;
    if (xyz[a] < g->origin[a] - 1e-9 * ext[a] || xyz[a] > g->origin[a] + ext[a] * (1 + 1e-9)) return TEM_EINVAL;
  }
  // nearest node plane in z
  int k = 0;
  {
    double z = g->origin[2], best = std::fabs(xyz[2] - z);
    for (int q2 = 0; q2 < nz; ++q2) {
      z += g->hz[q2];
      if (std::fabs(xyz[2] - z) < best) { best = std::fabs(xyz[2] - z); k = q2 + 1; }
    }
  }
  // bilinear weights between face centres (clamped to the outermost centres)
  auto weights = [](const std::vector<double>& h, double origin, double v, int* idx, double* w) {
    const int n = (int)h.size();
    std::vector<double> c(n);
    double x = origin;
    for (int q2 = 0; q2 < n; ++q2) { c[q2] = x + 0.5 * h[q2]; x += h[q2]; }
    if (v <= c[0]) { idx[0] = 0; w[0] = 1.0; return 1; }
    if (v >= c[n - 1]) { idx[0] = n - 1; w[0] = 1.0; return 1; }
    int a = 0;
    while (a + 1 < n && c[a + 1] <= v) ++a;
    const double t = (v - c[a]) / (c[a + 1] - c[a]);
    idx[0] = a; w[0] = 1.0 - t; idx[1] = a + 1; w[1] = t;
    return 2;
  };
  int ix[2], iy[2];
  double wx[2], wy[2];
  const int nxw = weights(g->hx, g->origin[0], xyz[0], ix, wx);
  const int nyw = weights(g->hy, g->origin[1], xyz[1], iy, wy);
  std::map<int64_t, double> acc;
  auto add = [&](int c, int i, int j, double w) {
    if (edge_valid_host(c, i, j, k, nx, ny, nz)) acc[edge_index(c, i, j, k, nx, ny, nz)] += w;
  };
  for (int a = 0; a < nxw; ++a)
    for (int b = 0; b < nyw; ++b) {
      const int i = ix[a], j = iy[b];
      const double w = wx[a] * wy[b];
      const double Lx = g->hx[i], Ly = g->hy[j];
      // d_t b_z = -circ / (Lx Ly),  circ = Lx e_x(i,j) + Ly e_y(i+1,j) - Lx e_x(i,j+1) - Ly e_y(i,j)
      add(0, i, j, -w / Ly);
      add(1, i + 1, j, -w / Lx);
      add(0, i, j + 1, w / Ly);
      add(1, i, j, w / Lx);
    }
  for (auto& kv : acc)
    if (kv.second != 0.0) q.push_back(Term{kv.first, kv.second});
  return TEM_OK;
}

}  // namespace tem
