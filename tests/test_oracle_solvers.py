"""Pins of the oracle's three solve routes and the forward model (Eq. (expm), (rmj), Sec. 3.3)."""
import numpy as np
import pytest

from oracle import rational as R
from oracle.solvers import solve_lu, solve_cocg
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W


@pytest.fixture(scope="module")
def small():
    m = W.uniform_model(8, 20.0, 3, 0.01, 80.0, 1e-5, 1e-3, 21, 16)
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    sh, c, err = R.tem_poles_residues(m.t, m.degree)
    return m, P, sh, c, err, P.dense()


def test_lu_matches_dense_solve(small):
    _, P, sh, _, _, _ = small
    A = P.K.toarray() - sh[0] * np.diag(P.Md)
    x, xd = solve_lu(P.K, P.Md, P.f, sh[0]), np.linalg.solve(A, P.f)
    # kappa(A) ~ 1e8 from curl-free modes in the air: x itself agrees only to ~kappa eps, but
    # both residuals are at rounding level and the receiver (a curl) sees none of those modes
    assert np.linalg.norm(A @ x - P.f) <= 1e-14 * np.linalg.norm(P.f)
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    assert np.abs(P.Q @ (x - xd)).max() <= 1e-10 * np.abs(P.Q @ xd).max()


def test_lu_rational_matches_eigenbasis(small):
    """T1 (LU per pole) and T0 (eigenbasis) evaluate the same rational function."""
    m, P, sh, c, _, eig = small
    d = P.forward(sh, c)
    d0 = np.stack([P.Q @ eig.rational(sh, c[:, k], P.f) for k in range(len(m.t))], axis=1)
    assert np.abs(d - d0).max() <= 1e-8 * np.abs(d).max()


def test_cocg_matches_lu(small):
    _, P, sh, _, _, _ = small
    for s in sh[[0, 3, 7]]:
        x, it, rel = solve_cocg(P.K, P.Md, P.f, s, tol=1e-13)
        assert rel <= 1e-13
        xl = solve_lu(P.K, P.Md, P.f, s)
        assert np.linalg.norm(x - xl) <= 1e-8 * np.linalg.norm(xl)


def test_conjugate_shift_gives_conjugate_solution(small):
    """K, M, f are real, so (K - conj(xi) M)^{-1} f = conj((K - xi M)^{-1} f)."""
    _, P, sh, _, _, _ = small
    x = solve_lu(P.K, P.Md, P.f, sh[2])
    xc = solve_lu(P.K, P.Md, P.f, np.conj(sh[2]))
    assert np.linalg.norm(xc - np.conj(x)) <= 1e-12 * np.linalg.norm(x)


def test_m_norm_error_bound(small):
    """Sec. 3.3: ||exp(-t A) b - r(A) b||_M <= ||b||_M max_x |exp(-t x) - r(x)| with A = M^{-1} K."""
    m, P, sh, c, err, eig = small
    b = P.f / P.Md
    bM = np.sqrt(b @ (P.Md * b))
    for k in range(len(m.t)):
        ex = eig.expm(m.t[k], P.f)
        ra = eig.rational(sh, c[:, k], P.f)
        gap = np.sqrt((ex - ra) @ (P.Md * (ex - ra)))
        assert gap <= bM * err * (1 + 1e-8) + 1e-14 * bM


def test_m_norm_decay(small):
    """Exact: d/dt (u^T M u) = -2 u^T K u <= 0, so ||u(t)||_M decreases; the rational
    family decreases up to 2 eps ||b||_M."""
    m, P, sh, c, err, eig = small
    b = P.f / P.Md
    bM = np.sqrt(b @ (P.Md * b))
    ex = [eig.expm(tk, P.f) for tk in m.t]
    ra = [eig.rational(sh, c[:, k], P.f) for k in range(len(m.t))]
    nrm = lambda u: np.sqrt(u @ (P.Md * u))
    ne, nr = [nrm(u) for u in ex], [nrm(u) for u in ra]
    # eigh leaves the (n-1)^3 curl-free modes at |lam| ~ 1e-15 lam_max instead of 0, so the
    # computed norm bottoms out at a rounding floor (~1e-10 ||b||_M here) instead of reaching 0
    floor = 1e-9 * bM
    assert all(ne[k + 1] <= ne[k] * (1 + 1e-12) + floor for k in range(len(ne) - 1))
    assert ne[0] > 1e3 * floor
    assert all(nr[k + 1] <= nr[k] + 2 * err * bM for k in range(len(nr) - 1))
    # the derivative identity itself, by a centred difference in t
    t, h = 2e-5, 1e-9
    up, um, u0 = eig.expm(t + h, P.f), eig.expm(t - h, P.f), eig.expm(t, P.f)
    lhs = (up @ (P.Md * up) - um @ (P.Md * um)) / (2 * h)
    rhs = -2.0 * (u0 @ (P.K @ u0))
    assert np.isclose(lhs, rhs, rtol=1e-4)


def test_forward_real_and_linear_in_current():
    m = W.uniform_model(6, 20.0, 2, 0.05, 40.0, 1e-5, 1e-3, 5, 8)
    sh, c, _ = R.tem_poles_residues(m.t, m.degree)
    P1 = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, current=1.0, origin=m.origin)
    P3 = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, current=3.0, origin=m.origin)
    assert np.allclose(P3.forward(sh, c), 3.0 * P1.forward(sh, c), rtol=1e-12)
