"""Oracle: shared-pole rational approximants to exp(-t x) on x >= 0 (FP64, NumPy).

Test infrastructure only (see ``oracle/__init__.py``).

What is computed (Section 3.2, Eq. (ratfam)-(rkfit)): one pole set xi_1..xi_m
shared by K rational functions r^[j](x) = sum_i alpha_i^[j] / (x - xi_i), each
approximating exp(-t_j x) for x >= 0.  The objective (Eq. (rkfit)) is the
weighted least-squares misfit sum_j w_j || r^[j](S) v - exp(-t_j S) v ||^2 with
S a diagonal surrogate whose eigenvalues densely sample [0, inf) and v all ones.
The paper gives the objective only; the iteration below is the RKFIT pole
relocation of Berljafa & Guettel (SISC 2017, Sec. 6.2) written for a diagonal
S, in real arithmetic so that complex poles stay in exact conjugate pairs:

  1. take the space spanned by 1 and 1/(x - xi_i) on the samples (a rational
     Krylov space with the current poles) and an orthonormal basis V of it;
  2. find the unit vector V c minimising sum_j w_j ||(I - V V^T) F_j V c||^2
     (smallest right singular vector of the stacked matrix);
  3. the roots of the rational function V c are the new poles.

After the last sweep the residues come from one linear least-squares fit per
time with the poles fixed (Eq. (ratfam)).  Times are normalised by t_max before
fitting and scaled back afterwards: poles xi/t_max, residues alpha/t_max.

Every function here is plain NumPy; nothing is blocked or fused.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "surrogate_samples", "initial_poles", "real_basis", "relocate_poles",
    "fit_residues", "rkfit", "evaluate", "uniform_error", "conj_reduce",
    "tem_poles_residues",
]


def surrogate_samples(tau_min: float, n: int = 2000) -> np.ndarray:
    """Eigenvalues of the diagonal surrogate S (Eq. (rkfit)): 0 plus a log grid.

    The grid spans [1e-2, 1e3 / tau_min]; beyond its top end exp(-tau x) is
    below exp(-1000) for every normalised time tau >= tau_min.
    """
    return np.concatenate(([0.0], np.logspace(-2.0, np.log10(1e3 / tau_min), n - 1)))


def initial_poles(m: int, tau_min: float) -> np.ndarray:
    """Starting poles: conjugate pairs -b/2 +- i b, b log-spaced on [1, 1/tau_min].

    An odd degree adds one real pole at -1.  (The paper does not give a
    starting guess; any set off [0, inf) serves RKFIT.)
    """
    npairs = m // 2
    b = np.logspace(0.0, np.log10(1.0 / tau_min), npairs) if npairs > 0 else np.zeros(0)
    poles = []
    for bk in b:
        poles += [complex(-0.5 * bk, bk), complex(-0.5 * bk, -bk)]
    if m % 2:
        poles.append(complex(-1.0, 0.0))
    return np.array(poles, dtype=np.complex128)


def _split(poles: np.ndarray, rtol: float = 1e-10):
    """Return (pair representatives with Im>0, real poles) of a conjugate-closed set."""
    re_mask = np.abs(poles.imag) <= rtol * np.maximum(np.abs(poles), 1e-300)
    real = np.sort(poles[re_mask].real)
    upper = poles[(~re_mask) & (poles.imag > 0)]
    upper = upper[np.argsort(np.abs(upper))]
    return upper, real


def real_basis(x: np.ndarray, poles: np.ndarray, const: bool) -> np.ndarray:
    """Columns [1], Re 1/(x-xi), Im 1/(x-xi) per pair, 1/(x-xi_r) per real pole."""
    upper, real = _split(poles)
    cols = [np.ones_like(x)] if const else []
    for xi in upper:
        g = 1.0 / (x - xi)
        cols += [g.real, g.imag]
    for xr in real:
        cols.append(1.0 / (x - xr))
    return np.stack(cols, axis=1)


def _zeros_of_real_form(c: np.ndarray, poles: np.ndarray) -> np.ndarray:
    """Roots of c0 + sum_pairs (c_re Re g + c_im Im g) + sum_real c_r/(x - xi_r).

    With g = 1/(x - a - ib) one has [Re g, -Im g] = (x I - A)^{-1} e_1 for
    A = [[a, b], [-b, a]], so the function is D + C (x I - A)^{-1} B with
    D = c0, C = [c_re, -c_im], B = e_1 per pair; its zeros are eig(A - B C / D).
    The matrix is real, so LAPACK returns exact conjugate pairs.
    """
    upper, real = _split(poles)
    n = 2 * len(upper) + len(real)
    A = np.zeros((n, n))
    B = np.zeros(n)
    C = np.zeros(n)
    pos = 1
    for blk, xi in enumerate(upper):
        a, b = xi.real, xi.imag
        r = 2 * blk
        A[r:r + 2, r:r + 2] = [[a, b], [-b, a]]
        B[r] = 1.0
        C[r], C[r + 1] = c[pos], -c[pos + 1]
        pos += 2
    off = 2 * len(upper)
    for q, xr in enumerate(real):
        A[off + q, off + q] = xr
        B[off + q] = 1.0
        C[off + q] = c[pos]
        pos += 1
    return np.linalg.eigvals(A - np.outer(B, C) / c[0])


def relocate_poles(x, tau, w, poles):
    """One RKFIT relocation sweep (steps 1-3 of the module docstring)."""
    Phi = real_basis(x, poles, const=True)
    V, R = np.linalg.qr(Phi)
    blocks = []
    for tj, wj in zip(tau, w):
        FV = np.exp(-tj * x)[:, None] * V
        blocks.append(np.sqrt(wj) * (FV - V @ (V.T @ FV)))
    _, _, vt = np.linalg.svd(np.vstack(blocks), full_matrices=False)
    c = np.linalg.solve(R, vt[-1])
    new = _zeros_of_real_form(c, poles)
    # keep the set conjugate-closed after rounding: snap near-real roots to the axis
    re_mask = np.abs(new.imag) <= 1e-10 * np.abs(new)
    new = np.where(re_mask, new.real + 0j, new)
    return new


def fit_residues(x, tau, poles):
    """Residues alpha[i, j] for fixed poles: one linear LSQ per time (Eq. (ratfam))."""
    Phi = real_basis(x, poles, const=False)
    F = np.exp(-np.outer(x, tau))
    coef, *_ = np.linalg.lstsq(Phi, F, rcond=None)
    upper, real = _split(poles)
    alpha = np.zeros((len(poles), len(tau)), dtype=np.complex128)
    xi = np.zeros(len(poles), dtype=np.complex128)
    pos = 0
    for p, z in enumerate(upper):
        a = (coef[pos] - 1j * coef[pos + 1]) / 2.0
        xi[2 * p], xi[2 * p + 1] = z, np.conj(z)
        alpha[2 * p], alpha[2 * p + 1] = a, np.conj(a)
        pos += 2
    off = 2 * len(upper)
    for q, z in enumerate(real):
        xi[off + q] = z
        alpha[off + q] = coef[pos]
        pos += 1
    return xi, alpha


def rkfit(tau, m, w=None, iters=12, nsamp=2000):
    """Shared-pole family for normalised times tau (max(tau) == 1).

    Returns (xi[m], alpha[m, K]) in the normalised variable.
    """
    tau = np.asarray(tau, dtype=np.float64)
    w = np.ones_like(tau) if w is None else np.asarray(w, dtype=np.float64)
    x = surrogate_samples(tau.min(), nsamp)
    poles = initial_poles(m, tau.min())
    best = None
    for _ in range(iters):
        poles = relocate_poles(x, tau, w, poles)
        xi, alpha = fit_residues(x, tau, poles)
        # the sweep can settle into a 2-cycle; keep the iterate with the
        # smallest weighted max misfit on the surrogate samples
        err = float((w * np.abs(np.exp(-np.outer(x, tau)) - evaluate(x, xi, alpha).real).max(axis=0)).max())
        if best is None or err < best[0]:
            best = (err, xi, alpha)
    return best[1], best[2]


def evaluate(x, xi, alpha):
    """r^[j](x) = sum_i alpha[i, j] / (x - xi_i) for every sample x and time j."""
    return (1.0 / (np.asarray(x)[:, None] - xi[None, :])) @ alpha


def uniform_error(tau, xi, alpha, w=None, xmax=None, n=20000):
    """Eq. (uniform_error): max_j w_j max_{x>=0} |exp(-tau_j x) - r^[j](x)| on a fine grid."""
    tau = np.asarray(tau)
    w = np.ones_like(tau) if w is None else np.asarray(w)
    if xmax is None:
        xmax = 1e4 / tau.min()
    x = np.concatenate(([0.0], np.logspace(-4.0, np.log10(xmax), n)))
    err = np.abs(np.exp(-np.outer(x, tau)) - evaluate(x, xi, alpha).real)
    per_t = err.max(axis=0)
    return float((w * per_t).max()), per_t


def conj_reduce(xi, alpha):
    """Eq. (rmj): keep one pole of each conjugate pair with weight 2, real poles with 1.

    Returns (shifts[s], c[s, K]) with sum_i alpha_i g(xi_i) = sum_k Re(c_k g(shift_k))
    for any g with g(conj z) = conj g(z).
    """
    upper_idx = [i for i in range(len(xi)) if xi[i].imag > 1e-10 * abs(xi[i])]
    real_idx = [i for i in range(len(xi)) if abs(xi[i].imag) <= 1e-10 * abs(xi[i])]
    shifts = np.array([xi[i] for i in upper_idx] + [xi[i].real + 0j for i in real_idx])
    c = np.array([2.0 * alpha[i] for i in upper_idx] + [alpha[i].real + 0j for i in real_idx])
    return shifts, c


def tem_poles_residues(t, m, w=None, iters=12, nsamp=2000):
    """Physical-time shifts and channel weights for the TEM forward model.

    t: channel times (s), strictly increasing.  Returns (shifts[s], c[s, K],
    uniform_err) where u(t_k) ~= sum_i Re(c[i, k] (K - shifts[i] M)^{-1} f).
    """
    t = np.asarray(t, dtype=np.float64)
    tmax = t.max()
    tau = t / tmax
    xi, alpha = rkfit(tau, m, w, iters=iters, nsamp=nsamp)
    err, _ = uniform_error(tau, xi, alpha, w)
    shifts, c = conj_reduce(xi, alpha)
    return shifts / tmax, c / tmax, err
