// tem_poles_residues: shared-pole rational family for exp(-t x) on x >= 0.
//
// Sec. 3.2, Eq. (ratfam)-(rkfit): one pole set xi_1..xi_m for K functions
// r^[j](x) = sum_i alpha_i^[j] / (x - xi_i) ~ exp(-t_j x), fitted by minimising
// sum_j w_j || r^[j](S) v - exp(-t_j S) v ||^2 over a diagonal surrogate S with
// eigenvalues densely sampling [0, inf) and v = ones.  The relocation step is
// the RKFIT one (Berljafa & Guettel 2017, Sec. 6.2) specialised to diagonal S:
//   V  = orthonormal basis of span{1, 1/(x - xi_i)} on the samples,
//   c  = argmin_{|c|=1} sum_j w_j |(I - V V^T) F_j V c|^2     (smallest right singular vector),
//   new poles = roots of the rational function V c.
// Everything runs in real arithmetic (a conjugate pair contributes the columns
// Re 1/(x - xi), Im 1/(x - xi)), so complex poles stay in exact pairs.  Times
// are normalised by t_max; poles and residues are scaled back by 1/t_max.
//
// Dense linear algebra (Householder QR, one-sided Jacobi SVD, Hessenberg
// reduction with Francis double-shift QR) is written out here: the sizes are
// tiny (<= 65 columns) and this runs once per channel set.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "../../include/tem.h"

namespace {

typedef std::complex<double> cd;

// Column-major dense matrix.
struct Mat {
  int m = 0, n = 0;
  std::vector<double> a;
  Mat() {}
  Mat(int m_, int n_) : m(m_), n(n_), a((size_t)m_ * n_, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)j * m + i]; }
  double operator()(int i, int j) const { return a[(size_t)j * m + i]; }
};

// Householder QR of A (m >= n), in place: R in the upper triangle, the
// reflectors' vectors below it with their scalars in tau.
void householder_qr(Mat& A, std::vector<double>& tau) {
  const int m = A.m, n = A.n;
  tau.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += A(i, k) * A(i, k);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double alpha = A(k, k) > 0 ? -nrm : nrm;
    const double v0 = A(k, k) - alpha;
    // v = [1, A(k+1:,k)/v0], tau = -v0/alpha
    for (int i = k + 1; i < m; ++i) A(i, k) /= v0;
    tau[k] = -v0 / alpha;
    A(k, k) = alpha;
    for (int j = k + 1; j < n; ++j) {
      double s = A(k, j);
      for (int i = k + 1; i < m; ++i) s += A(i, k) * A(i, j);
      s *= tau[k];
      A(k, j) -= s;
      for (int i = k + 1; i < m; ++i) A(i, j) -= s * A(i, k);
    }
  }
}

// Apply Q^T (from householder_qr) to the columns of B.
void apply_qt(const Mat& A, const std::vector<double>& tau, Mat& B) {
  for (int k = 0; k < A.n; ++k) {
    if (tau[k] == 0.0) continue;
    for (int j = 0; j < B.n; ++j) {
      double s = B(k, j);
      for (int i = k + 1; i < A.m; ++i) s += A(i, k) * B(i, j);
      s *= tau[k];
      B(k, j) -= s;
      for (int i = k + 1; i < A.m; ++i) B(i, j) -= s * A(i, k);
    }
  }
}

// Thin Q (m x n) from householder_qr.
Mat form_q(const Mat& A, const std::vector<double>& tau) {
  Mat Q(A.m, A.n);
  for (int j = 0; j < A.n; ++j) Q(j, j) = 1.0;
  for (int k = A.n - 1; k >= 0; --k) {
    if (tau[k] == 0.0) continue;
    for (int j = 0; j < A.n; ++j) {
      double s = Q(k, j);
      for (int i = k + 1; i < A.m; ++i) s += A(i, k) * Q(i, j);
      s *= tau[k];
      Q(k, j) -= s;
      for (int i = k + 1; i < A.m; ++i) Q(i, j) -= s * A(i, k);
    }
  }
  return Q;
}

// Solve R x = b (R upper triangular, the leading n x n of A).
std::vector<double> back_substitute(const Mat& A, std::vector<double> b) {
  const int n = A.n;
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A(i, j) * b[j];
    b[i] = A(i, i) != 0.0 ? s / A(i, i) : 0.0;
  }
  return b;
}

// Right singular vector of the smallest singular value of the n x n matrix R
// (one-sided Jacobi: rotate column pairs of R until orthogonal, accumulating V).
std::vector<double> smallest_right_singular_vector(Mat R) {
  const int n = R.n;
  Mat V(n, n);
  for (int i = 0; i < n; ++i) V(i, i) = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0, beta = 0, gamma = 0;
        for (int i = 0; i < R.m; ++i) {
          alpha += R(i, p) * R(i, p);
          beta += R(i, q) * R(i, q);
          gamma += R(i, p) * R(i, q);
        }
        if (gamma == 0.0) continue;
        off = std::max(off, std::fabs(gamma) / std::sqrt(alpha * beta));
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < R.m; ++i) {
          const double a = R(i, p), b = R(i, q);
          R(i, p) = c * a - s * b;
          R(i, q) = s * a + c * b;
        }
        for (int i = 0; i < n; ++i) {
          const double a = V(i, p), b = V(i, q);
          V(i, p) = c * a - s * b;
          V(i, q) = s * a + c * b;
        }
      }
    if (off < 1e-15) break;
  }
  int best = 0;
  double bs = 1e300;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < R.m; ++i) s += R(i, j) * R(i, j);
    if (s < bs) { bs = s; best = j; }
  }
  std::vector<double> v(n);
  for (int i = 0; i < n; ++i) v[i] = V(i, best);
  return v;
}

// Eigenvalues of a real n x n matrix (row-major H): Householder reduction to
// upper Hessenberg form, then Francis double-shift QR steps with deflation
// (Golub & Van Loan, Sec. 7.4-7.5).  Complex eigenvalues come in exact pairs.
bool real_eigenvalues(std::vector<double> H, int n, std::vector<cd>& eig) {
  auto at = [&](int i, int j) -> double& { return H[(size_t)i * n + j]; };
  // Hessenberg reduction
  for (int k = 0; k < n - 2; ++k) {
    double nrm = 0;
    for (int i = k + 1; i < n; ++i) nrm += at(i, k) * at(i, k);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    std::vector<double> v(n, 0.0);
    const double alpha = at(k + 1, k) > 0 ? -nrm : nrm;
    for (int i = k + 1; i < n; ++i) v[i] = at(i, k);
    v[k + 1] -= alpha;
    double vv = 0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = 0; j < n; ++j) {  // H = P H
      double s = 0;
      for (int i = k + 1; i < n; ++i) s += v[i] * at(i, j);
      s *= 2.0 / vv;
      for (int i = k + 1; i < n; ++i) at(i, j) -= s * v[i];
    }
    for (int i = 0; i < n; ++i) {  // H = H P
      double s = 0;
      for (int j = k + 1; j < n; ++j) s += at(i, j) * v[j];
      s *= 2.0 / vv;
      for (int j = k + 1; j < n; ++j) at(i, j) -= s * v[j];
    }
    for (int i = k + 2; i < n; ++i) at(i, k) = 0.0;
  }
  double anorm = 0;
  for (double x : H) anorm = std::max(anorm, std::fabs(x));
  const double eps = 2.220446049250313e-16;
  eig.clear();
  int hi = n - 1, iter = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      double s = std::fabs(at(l - 1, l - 1)) + std::fabs(at(l, l));
      if (s == 0.0) s = anorm;
      if (std::fabs(at(l, l - 1)) <= eps * s) {
        at(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {
      eig.push_back(cd(at(hi, hi), 0.0));
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {
      const double a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
      const double p = 0.5 * (a - d), disc = p * p + b * c, mid = 0.5 * (a + d);
      if (disc >= 0.0) {
        const double sq = std::sqrt(disc);
        const double r1 = mid + (p >= 0 ? sq : -sq);
        const double r2 = r1 != 0.0 ? (a * d - b * c) / r1 : mid - (p >= 0 ? sq : -sq);
        eig.push_back(cd(r1, 0.0));
        eig.push_back(cd(r2, 0.0));
      } else {
        const double sq = std::sqrt(-disc);
        eig.push_back(cd(mid, sq));
        eig.push_back(cd(mid, -sq));
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++total > 100 * n) return false;
    ++iter;
    double tr, det;
    if (iter % 10 == 0) {  // exceptional shift
      const double s = std::fabs(at(hi, hi - 1)) + std::fabs(at(hi - 1, hi - 2));
      tr = 1.5 * s;
      det = s * s;
    } else {
      tr = at(hi - 1, hi - 1) + at(hi, hi);
      det = at(hi - 1, hi - 1) * at(hi, hi) - at(hi - 1, hi) * at(hi, hi - 1);
    }
    // first column of (H - s1 I)(H - s2 I) on the active block
    double x = at(l, l) * at(l, l) + at(l, l + 1) * at(l + 1, l) - tr * at(l, l) + det;
    double y = at(l + 1, l) * (at(l, l) + at(l + 1, l + 1) - tr);
    double z = at(l + 1, l) * at(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      // reflector P = I - 2 v v^T / v^T v with P (x, y, z)^T = (*, 0, 0)^T
      const double nrm = std::sqrt(x * x + y * y + z * z);
      if (nrm != 0.0) {
        const double alpha = x > 0 ? -nrm : nrm;
        const double v0 = x - alpha, v1 = y, v2 = z;
        const double vv = v0 * v0 + v1 * v1 + v2 * v2;
        const int c0 = std::max(l, k - 1);
        for (int j = c0; j <= hi; ++j) {
          const double s = 2.0 * (v0 * at(k, j) + v1 * at(k + 1, j) + v2 * at(k + 2, j)) / vv;
          at(k, j) -= s * v0;
          at(k + 1, j) -= s * v1;
          at(k + 2, j) -= s * v2;
        }
        const int r1 = std::min(hi, k + 3);
        for (int i = l; i <= r1; ++i) {
          const double s = 2.0 * (at(i, k) * v0 + at(i, k + 1) * v1 + at(i, k + 2) * v2) / vv;
          at(i, k) -= s * v0;
          at(i, k + 1) -= s * v1;
          at(i, k + 2) -= s * v2;
        }
      }
      x = at(k + 1, k);
      y = at(k + 2, k);
      if (k < hi - 2) z = at(k + 3, k);
    }
    // last 2-vector
    {
      const int k = hi - 1;
      const double nrm = std::sqrt(x * x + y * y);
      if (nrm != 0.0) {
        const double alpha = x > 0 ? -nrm : nrm;
        const double v0 = x - alpha, v1 = y;
        const double vv = v0 * v0 + v1 * v1;
        for (int j = std::max(l, k - 1); j <= hi; ++j) {
          const double s = 2.0 * (v0 * at(k, j) + v1 * at(k + 1, j)) / vv;
          at(k, j) -= s * v0;
          at(k + 1, j) -= s * v1;
        }
        for (int i = l; i <= hi; ++i) {
          const double s = 2.0 * (at(i, k) * v0 + at(i, k + 1) * v1) / vv;
          at(i, k) -= s * v0;
          at(i, k + 1) -= s * v1;
        }
      }
    }
  }
  return true;
}

// ---------------------------------------------------------------- the fit
struct PoleSet {
  std::vector<cd> upper;     // one pole of each conjugate pair (Im > 0), by |xi|
  std::vector<double> real;  // real poles, ascending
  int degree() const { return 2 * (int)upper.size() + (int)real.size(); }
};

PoleSet classify(const std::vector<cd>& z) {
  PoleSet P;
  for (const cd& v : z) {
    if (std::fabs(v.imag()) <= 1e-10 * std::abs(v)) P.real.push_back(v.real());
    else if (v.imag() > 0) P.upper.push_back(v);
  }
  std::sort(P.upper.begin(), P.upper.end(), [](const cd& a, const cd& b) { return std::abs(a) < std::abs(b); });
  std::sort(P.real.begin(), P.real.end());
  return P;
}

std::vector<double> logspace(double a, double b, int n) {
  std::vector<double> x(n);
  const double step = n > 1 ? (b - a) / (n - 1) : 0.0;
  for (int i = 0; i < n; ++i) x[i] = std::pow(10.0, a + i * step);
  if (n > 1) x[n - 1] = std::pow(10.0, b);
  return x;
}

// Columns [1], Re g, Im g per pair, 1/(x - xi_r) per real pole.
Mat basis(const std::vector<double>& x, const PoleSet& P, bool with_const) {
  const int m = (int)x.size();
  Mat B(m, (with_const ? 1 : 0) + P.degree());
  int col = 0;
  if (with_const) {
    for (int i = 0; i < m; ++i) B(i, 0) = 1.0;
    col = 1;
  }
  for (const cd& xi : P.upper) {
    for (int i = 0; i < m; ++i) {
      const cd g = 1.0 / (cd(x[i], 0.0) - xi);
      B(i, col) = g.real();
      B(i, col + 1) = g.imag();
    }
    col += 2;
  }
  for (double xr : P.real) {
    for (int i = 0; i < m; ++i) B(i, col) = 1.0 / (x[i] - xr);
    ++col;
  }
  return B;
}

// One relocation sweep; returns false if the eigen-solve fails.
bool relocate(const std::vector<double>& x, const std::vector<double>& tau, const std::vector<double>& w,
              PoleSet& P) {
  Mat Phi = basis(x, P, true);
  std::vector<double> tq;
  householder_qr(Phi, tq);
  Mat V = form_q(Phi, tq);
  const int L = V.m, n = V.n, K = (int)tau.size();
  Mat S((size_t)L * K > 0 ? L * K : 1, n);
  std::vector<double> f(L);
  for (int j = 0; j < K; ++j) {
    const double sw = std::sqrt(w[j]);
    for (int i = 0; i < L; ++i) f[i] = std::exp(-tau[j] * x[i]);
    // FV = diag(f) V;  block = FV - V (V^T FV)
    std::vector<double> VtFV((size_t)n * n, 0.0);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double s = 0;
        for (int i = 0; i < L; ++i) s += V(i, a) * f[i] * V(i, b);
        VtFV[(size_t)b * n + a] = s;
      }
    for (int b = 0; b < n; ++b)
      for (int i = 0; i < L; ++i) {
        double s = f[i] * V(i, b);
        for (int a = 0; a < n; ++a) s -= V(i, a) * VtFV[(size_t)b * n + a];
        S(j * L + i, b) = sw * s;
      }
  }
  std::vector<double> ts;
  householder_qr(S, ts);
  Mat R(n, n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= j; ++i) R(i, j) = S(i, j);
  std::vector<double> cv = smallest_right_singular_vector(R);
  std::vector<double> c = back_substitute(Phi, cv);  // coefficients in the Phi basis
  if (c[0] == 0.0) return false;
  // zeros of D + C (x I - A)^{-1} B: eig(A - B C / D); per pair A = [[a, b], [-b, a]],
  // B = e1, C = [c_re, -c_im]; per real pole A = [xi], B = 1, C = [c_r]
  const int m = P.degree();
  std::vector<double> A((size_t)m * m, 0.0), Bv(m, 0.0), Cv(m, 0.0);
  int pos = 1, r = 0;
  for (const cd& xi : P.upper) {
    A[(size_t)r * m + r] = xi.real();
    A[(size_t)r * m + r + 1] = xi.imag();
    A[(size_t)(r + 1) * m + r] = -xi.imag();
    A[(size_t)(r + 1) * m + r + 1] = xi.real();
    Bv[r] = 1.0;
    Cv[r] = c[pos];
    Cv[r + 1] = -c[pos + 1];
    pos += 2;
    r += 2;
  }
  for (double xr : P.real) {
    A[(size_t)r * m + r] = xr;
    Bv[r] = 1.0;
    Cv[r] = c[pos];
    ++pos;
    ++r;
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] -= Bv[i] * Cv[j] / c[0];
  std::vector<cd> z;
  if (!real_eigenvalues(A, m, z)) return false;
  PoleSet Q = classify(z);
  if (Q.degree() != m) return false;
  P = Q;
  return true;
}

// Residues for fixed poles: one LSQ per time; alpha[(pole)][j] complex (upper pairs then reals).
void fit_residues(const std::vector<double>& x, const std::vector<double>& tau, const PoleSet& P,
                  std::vector<cd>& alpha) {
  Mat Phi = basis(x, P, false);
  const int L = Phi.m, n = Phi.n, K = (int)tau.size();
  std::vector<double> tq;
  householder_qr(Phi, tq);
  Mat F(L, K);
  for (int j = 0; j < K; ++j)
    for (int i = 0; i < L; ++i) F(i, j) = std::exp(-tau[j] * x[i]);
  apply_qt(Phi, tq, F);
  const int npole = (int)P.upper.size() + (int)P.real.size();
  alpha.assign((size_t)npole * K, cd(0, 0));
  for (int j = 0; j < K; ++j) {
    std::vector<double> b(n);
    for (int i = 0; i < n; ++i) b[i] = F(i, j);
    std::vector<double> coef = back_substitute(Phi, b);
    int pos = 0, p = 0;
    for (size_t u = 0; u < P.upper.size(); ++u, ++p) {
      alpha[(size_t)p * K + j] = cd(coef[pos], -coef[pos + 1]) * 0.5;
      pos += 2;
    }
    for (size_t u = 0; u < P.real.size(); ++u, ++p) {
      alpha[(size_t)p * K + j] = cd(coef[pos], 0.0);
      ++pos;
    }
  }
}

// max_j w_j max_x |exp(-tau_j x) - r^[j](x)| on the given samples
double max_error(const std::vector<double>& x, const std::vector<double>& tau, const std::vector<double>& w,
                 const PoleSet& P, const std::vector<cd>& alpha) {
  const int K = (int)tau.size();
  double worst = 0.0;
  for (int j = 0; j < K; ++j) {
    double e = 0.0;
    for (double xv : x) {
      double r = 0.0;
      int p = 0;
      for (const cd& xi : P.upper) {
        r += 2.0 * (alpha[(size_t)p * K + j] / (cd(xv, 0.0) - xi)).real();
        ++p;
      }
      for (double xr : P.real) {
        r += alpha[(size_t)p * K + j].real() / (xv - xr);
        ++p;
      }
      e = std::max(e, std::fabs(std::exp(-tau[j] * xv) - r));
    }
    worst = std::max(worst, w[j] * e);
  }
  return worst;
}

}  // namespace

extern "C" int tem_poles_residues(const double* t, int64_t K, int64_t degree, const double* weights,
                                  double* xi_out, double* c_out, int64_t* s_out, double* uniform_err_out) {
  if (!t || !xi_out || !c_out || !s_out || K < 1 || K > 10000 || degree < 1 || degree > 64) return TEM_EINVAL;
  for (int64_t k = 0; k < K; ++k) {
    if (!(std::isfinite(t[k]) && t[k] > 0.0)) return TEM_EINVAL;
    if (k > 0 && !(t[k] > t[k - 1])) return TEM_EINVAL;
    if (weights && !(std::isfinite(weights[k]) && weights[k] > 0.0)) return TEM_EINVAL;
  }
  const double tmax = t[K - 1];
  std::vector<double> tau(K), w(K, 1.0);
  for (int64_t k = 0; k < K; ++k) {
    tau[k] = t[k] / tmax;
    if (weights) w[k] = weights[k];
  }
  const double tau_min = tau[0];
  // surrogate eigenvalues: 0 and a log grid on [1e-2, 1e3 / tau_min]
  std::vector<double> x = logspace(-2.0, std::log10(1e3 / tau_min), 1999);
  x.insert(x.begin(), 0.0);
  // starting poles: pairs -b/2 +- i b, b log-spaced on [1, 1/tau_min]; odd degree adds -1
  PoleSet P;
  const int npairs = int(degree / 2);
  if (npairs > 0) {
    std::vector<double> b = logspace(0.0, std::log10(1.0 / tau_min), npairs);
    for (double bk : b) P.upper.push_back(cd(-0.5 * bk, bk));
  }
  if (degree % 2) P.real.push_back(-1.0);
  P = classify([&] {
    std::vector<cd> z;
    for (auto& u : P.upper) { z.push_back(u); z.push_back(std::conj(u)); }
    for (double r : P.real) z.push_back(cd(r, 0));
    return z;
  }());
  double best = 1e300;
  PoleSet bestP;
  std::vector<cd> bestA;
  for (int it = 0; it < 12; ++it) {
    if (!relocate(x, tau, w, P)) break;
    std::vector<cd> alpha;
    fit_residues(x, tau, P, alpha);
    const double e = max_error(x, tau, w, P, alpha);
    if (std::isfinite(e) && e < best) {
      best = e;
      bestP = P;
      bestA = alpha;
    }
  }
  if (bestA.empty()) return TEM_EINVAL;
  // The poles must stay off [0, inf), the spectrum of M^{-1} K (Sec. 3.2).  A fit that has
  // saturated (uniform error near rounding) can leave spurious real poles there, doublets
  // with residues at rounding level: drop them and refit the residues on the others.
  {
    std::vector<double> keep;
    for (double r : bestP.real)
      if (r < 0.0) keep.push_back(r);
    if (keep.size() != bestP.real.size()) {
      bestP.real = keep;
      if (bestP.upper.empty() && bestP.real.empty()) return TEM_EINVAL;
      bestA.clear();
      fit_residues(x, tau, bestP, bestA);
    }
  }
  // shifts: pairs (Im > 0) then real poles; c = 2 alpha for pairs, alpha for real poles
  const int s = (int)bestP.upper.size() + (int)bestP.real.size();
  int p = 0;
  for (const cd& z : bestP.upper) {
    xi_out[2 * p] = z.real() / tmax;
    xi_out[2 * p + 1] = z.imag() / tmax;
    for (int64_t k = 0; k < K; ++k) {
      const cd a = 2.0 * bestA[(size_t)p * K + k] / tmax;
      c_out[2 * (p * K + k)] = a.real();
      c_out[2 * (p * K + k) + 1] = a.imag();
    }
    ++p;
  }
  for (double r : bestP.real) {
    xi_out[2 * p] = r / tmax;
    xi_out[2 * p + 1] = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      c_out[2 * (p * K + k)] = bestA[(size_t)p * K + k].real() / tmax;
      c_out[2 * (p * K + k) + 1] = 0.0;
    }
    ++p;
  }
  *s_out = s;
  if (uniform_err_out) {
    std::vector<double> xf = logspace(-4.0, std::log10(1e4 / tau_min), 20000);
    xf.insert(xf.begin(), 0.0);
    *uniform_err_out = max_error(xf, tau, w, bestP, bestA);
  }
  return TEM_OK;
}
