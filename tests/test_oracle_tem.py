"""Pins of the oracle's physics and adjoint: halfspace closed form, its limits, finite differences."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import halfspace as H
from oracle import rational as R
from oracle.tem import TEMProblem
from oracle.yee import MU0
from paper_2506_11657_gb300 import workloads as W


def test_halfspace_late_time_limit():
    """Sec. 5.2: d_t b_z decays as t^{-5/2}; the closed form must reach its asymptote."""
    t = np.array([1e-1, 1.0, 10.0])
    r = H.dbzdt_central_loop(t, 0.01, 30.0) / H.late_time_dbzdt(t, 0.01, 30.0)
    assert np.allclose(r, 1.0, rtol=2e-3)
    assert abs(r[2] - 1) < abs(r[0] - 1)


def test_halfspace_early_time_limit():
    """t -> 0+: the bracket tends to 3, so d_t b_z -> -3 I / (sigma a^3)."""
    v = H.dbzdt_central_loop(np.array([1e-12]), 0.1, 5.0, current=2.0)[0]
    assert np.isclose(v, -3.0 * 2.0 / (0.1 * 125.0), rtol=1e-9)


def test_halfspace_integrates_to_dc_field():
    """int_0^inf d_t b_z dt = b_z(inf) - b_z(0+) = -mu0 I / (2 a): the static field at the
    centre of a loop, which the ground currents hold at t = 0+."""
    a, s, I = 40.0, 0.02, 1.5
    f = lambda lt: H.dbzdt_central_loop(np.exp(lt), s, a, I) * np.exp(lt)
    val, _ = quad(f, np.log(1e-12), np.log(1e4), limit=400)
    assert np.isclose(val, -MU0 * I / (2 * a), rtol=1e-6)


@pytest.mark.slow_cpu
def test_tiny16_matches_halfspace_early_channels():
    """Physics check (not parity): the 16^3 model against the closed form with the loop's
    equal-area radius.  The 320 m Dirichlet box truncates diffusion later on, so only
    channels up to 2.5e-5 s are compared, within 15 %."""
    m = W.tiny16()
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    sh, c, _ = R.tem_poles_residues(m.t, m.degree)
    d = P.forward(sh, c)[0]
    side = m.loop_xy[1, 0] - m.loop_xy[0, 0]
    hs = H.dbzdt_central_loop(m.t, 0.01, side / np.sqrt(np.pi))
    early = m.t <= 2.6e-5
    assert np.all(d[early] < 0)
    assert np.all(np.abs(d[early] / hs[early] - 1) < 0.15)


def test_adjoint_matches_finite_differences():
    """The adjoint gradient (Sec. 4) against central differences of the forward in log sigma."""
    m = W.uniform_model(6, 20.0, 2, 0.02, 40.0, 1e-5, 1e-3, 7, 8)
    rng = np.random.default_rng(11)
    sigma = m.sigma * np.where(m.sigma > 1e-6, 10 ** rng.uniform(-0.5, 0.5, m.sigma.shape), 1.0)
    rx = np.array([[0.0, 0.0, 0.0], [10.0, -5.0, 0.0]])
    sh, c, _ = R.tem_poles_residues(m.t, m.degree)
    P = TEMProblem(m.hx, m.hy, m.hz, sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    d = P.forward(sh, c)
    gres = rng.standard_normal(d.shape) / np.abs(d).mean()
    g = P.adjoint_gradient(sh, c, gres)
    cells = rng.choice(np.flatnonzero(sigma.ravel() > 1e-6), 6, replace=False)
    cells = np.concatenate((cells, np.flatnonzero(sigma.ravel() < 1e-6)[:2]))
    delta = 1e-4
    for cidx in cells:
        sp_, sm_ = sigma.ravel().copy(), sigma.ravel().copy()
        sp_[cidx] *= np.exp(delta)
        sm_[cidx] *= np.exp(-delta)
        dp = TEMProblem(m.hx, m.hy, m.hz, sp_, m.loop_xy, m.z_loop, rx, origin=m.origin).forward(sh, c)
        dm = TEMProblem(m.hx, m.hy, m.hz, sm_, m.loop_xy, m.z_loop, rx, origin=m.origin).forward(sh, c)
        fd = ((dp - dm) * gres).sum() / (2 * delta)
        assert abs(fd - g[cidx]) <= 1e-5 * np.abs(g).max() + 1e-6 * abs(fd), (cidx, fd, g[cidx])


def _jvp_model():
    m = W.uniform_model(6, 20.0, 2, 0.02, 40.0, 1e-5, 1e-3, 7, 8)
    rng = np.random.default_rng(12)
    sigma = m.sigma * np.where(m.sigma > 1e-6, 10 ** rng.uniform(-0.5, 0.5, m.sigma.shape), 1.0)
    rx = np.array([[0.0, 0.0, 0.0], [10.0, -5.0, 0.0], [-20.0, 15.0, 0.0]])
    sh, c, _ = R.tem_poles_residues(m.t, m.degree)
    return m, sigma, rx, sh, c, rng


def test_jvp_matches_directional_finite_differences():
    """J dm (Sec. 4) against central differences of the forward along a random direction in
    log sigma: (d(m + h dm) - d(m - h dm)) / 2h, h = 1e-4 (truncation O(h^2))."""
    m, sigma, rx, sh, c, rng = _jvp_model()
    P = TEMProblem(m.hx, m.hy, m.hz, sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    dm = rng.standard_normal(sigma.size)
    jd = P.jvp(sh, c, dm)
    h = 1e-4
    dp = TEMProblem(m.hx, m.hy, m.hz, sigma.ravel() * np.exp(h * dm), m.loop_xy, m.z_loop, rx,
                    origin=m.origin).forward(sh, c)
    dn = TEMProblem(m.hx, m.hy, m.hz, sigma.ravel() * np.exp(-h * dm), m.loop_xy, m.z_loop, rx,
                    origin=m.origin).forward(sh, c)
    fd = (dp - dn) / (2 * h)
    assert np.abs(fd - jd).max() <= 1e-6 * np.abs(jd).max()
    # a direction confined to the air cells moves the response much less than one in the earth
    air = (sigma.ravel() < 1e-6).astype(float)
    assert np.abs(P.jvp(sh, c, air)).max() < 1e-3 * np.abs(P.jvp(sh, c, 1.0 - air)).max()


def test_jvp_is_the_transpose_of_the_adjoint():
    """<g, J dm> = <J^T g, dm> with the separately pinned adjoint gradient."""
    m, sigma, rx, sh, c, rng = _jvp_model()
    P = TEMProblem(m.hx, m.hy, m.hz, sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    d, xs = P.forward(sh, c, return_solutions=True)
    dm = rng.standard_normal(sigma.size)
    g = rng.standard_normal(d.shape)
    lhs = np.sum(g * P.jvp(sh, c, dm, xs=xs))
    rhs = np.dot(P.adjoint_gradient(sh, c, g, xs=xs), dm)
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs(rhs))


def test_jvp_on_random_widths_matches_finite_differences():
    """J dm on a grid of unequal cell widths against central differences of the forward."""
    rng = np.random.default_rng(13)
    nx, ny, nz, air = 6, 5, 7, 2
    hx, hy, hz = rng.uniform(10, 30, nx), rng.uniform(10, 30, ny), rng.uniform(10, 30, nz)
    xn = np.concatenate(([0.0], np.cumsum(hx))) - hx[:3].sum()
    yn = np.concatenate(([0.0], np.cumsum(hy))) - hy[:2].sum()
    origin = (-hx[:3].sum(), -hy[:2].sum(), -hz[:nz - air].sum())
    sigma = np.full((nz, ny, nx), 1e-8)
    sigma[:nz - air] = 10 ** rng.uniform(-2.5, -1.0, (nz - air, ny, nx))
    loop = np.array([[xn[2], yn[1]], [xn[4], yn[1]], [xn[4], yn[3]], [xn[2], yn[3]]])
    rx = np.array([[xn[3], yn[2], 0.0], [0.5 * (xn[1] + xn[2]), 0.3 * yn[3] + 0.7 * yn[4], 0.0]])
    t = np.logspace(-5, -3, 6)
    sh, c, _ = R.tem_poles_residues(t, 8)
    P = TEMProblem(hx, hy, hz, sigma, loop, 0.0, rx, origin=origin)
    dm = rng.standard_normal(sigma.size) * (sigma.ravel() > 1e-6)
    jd = P.jvp(sh, c, dm)
    h = 1e-4
    dp = TEMProblem(hx, hy, hz, sigma.ravel() * np.exp(h * dm), loop, 0.0, rx, origin=origin).forward(sh, c)
    dn = TEMProblem(hx, hy, hz, sigma.ravel() * np.exp(-h * dm), loop, 0.0, rx, origin=origin).forward(sh, c)
    assert np.abs((dp - dn) / (2 * h) - jd).max() <= 1e-6 * np.abs(jd).max()
