"""Forward parity on grids with non-uniform cell widths, where the solver's stencil reads a
different L, L* and 1/L for every column and plane (on uniform grids an index slip in that
geometry would cancel out):

* a small grid with random widths in x, y and z and a blocky earth, FP64 and mixed, against
  the oracle's sparse-LU response with the per-channel bound of the forward tests;
* the adjoint gradient and J dm on the random-width grid against the oracle (FP64);
* the padded layered model (48^3 core of 10 m cells, 8 padding cells growing by 1.15 on every
  side), mixed precision as the benchmark runs it: every FP64 solution solves the oracle's own
  assembled system to 1e-11 and the response is the oracle's combination of the solutions.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W
from tests._layout import lib_index_of_interior

pytestmark = pytest.mark.gpu


def _random_width_model():
    rng = np.random.default_rng(51)
    nx, ny, nz, air = 18, 15, 20, 5
    hx, hy, hz = rng.uniform(6.0, 16.0, nx), rng.uniform(6.0, 16.0, ny), rng.uniform(6.0, 16.0, nz)
    _, xn0 = W._centres(hx, 0.0)
    _, yn0 = W._centres(hy, 0.0)
    origin = (-xn0[nx // 2], -yn0[ny // 2], -hz[: nz - air].sum())
    _, xn = W._centres(hx, origin[0])
    _, yn = W._centres(hy, origin[1])
    sigma = W._block_sigma(nz, ny, nx, air, 4, rng, (0.5, 2.5))
    loop = W._square_loop(60.0, xn, yn)
    # two receivers on nodes, two between nodes (bilinear weights over unequal z faces)
    rx = np.array([[0.0, 0.0, 0.0], [xn[nx // 2 + 3], yn[ny // 2 - 2], 0.0], [xn[3], yn[ny - 4], 0.0],
                   [0.37 * xn[nx // 2 + 2] + 0.63 * xn[nx // 2 + 3], 0.8 * yn[ny // 2 - 3] + 0.2 * yn[ny // 2 - 2], 0.0],
                   [0.5 * (xn[2] + xn[3]), 0.25 * yn[ny - 5] + 0.75 * yn[ny - 4], 0.0]])
    return W.Model("randwidth", hx, hy, hz, origin, sigma, loop, 0.0, rx, W.channel_times(1e-5, 1e-2, 10), 12)


@pytest.fixture(scope="module")
def small():
    m = _random_width_model()
    shifts, c, _ = R.tem_poles_residues(m.t, m.degree)
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    d, xs = P.forward(shifts, c, return_solutions=True)
    y = np.stack([P.Q @ x for x in xs])
    S = np.einsum("ik,ir->rk", np.abs(c), np.abs(y))
    return m, shifts, c, d, S


@pytest.mark.parametrize("prec,rel,floor", [("fp64", 1e-6, 1e-10), ("mixed", 1e-5, 1e-9)])
def test_random_widths_match_oracle(small, prec, rel, floor):
    from paper_2506_11657_gb300 import tem
    m, shifts, c, d, S = small
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    opt = tem.default_options(precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, opt)
    assert res.status == tem.TEM_OK
    from tests._parity import check
    check(res.d, d, S, rel, floor, f"random widths {prec}")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_padded_layered_model_solves_the_oracle_system(prec):
    """The padded layered model (64^3 with geometric padding) in plain FP64 COCG and in mixed
    precision: every FP64 solution solves the oracle's assembled system to 1e-11."""
    from paper_2506_11657_gb300 import tem
    m = W.layered64()
    shifts, c, _ = tem.poles_residues(m.t, m.degree)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, tem.default_options(precision=prec),
                      keep_state=True)
    assert res.status == tem.TEM_OK
    xs = [res.state.solution(i) for i in range(len(shifts))]
    res.state.close()
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    idx = lib_index_of_interior(P.grid)
    nf = np.linalg.norm(P.f)
    ys = []
    for i, x in enumerate(xs):
        xi = x[idx]
        r = P.f - (P.K @ xi - shifts[i] * (P.Md * xi))
        assert np.linalg.norm(r) / nf <= 1e-11, (i, np.linalg.norm(r) / nf)
        ys.append(P.Q @ xi)
    y = np.stack(ys)
    d_ref = np.einsum("ik,ir->rk", c, y).real
    S = np.einsum("ik,ir->rk", np.abs(c), np.abs(y))
    assert np.all(np.abs(res.d - d_ref) <= 1e-12 * S + 1e-300)


def test_random_widths_adjoint_and_jvp_match_oracle(small):
    """The adjoint gradient and J dm weight by sigma_c V_c / 4 with per-axis widths: both against
    the oracle (FP64 solves to 1e-13), relative to their largest entries."""
    from paper_2506_11657_gb300 import tem
    m, shifts, c, d, S = small
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    _, xs = P.forward(shifts, c, return_solutions=True)
    rng = np.random.default_rng(52)
    g = rng.standard_normal(d.shape) / np.abs(d).mean()
    dm = rng.standard_normal(m.sigma.size) * (m.sigma.ravel() > 1e-6)
    grad_ref = P.adjoint_gradient(shifts, c, g, xs=xs)
    jd_ref = P.jvp(shifts, c, dm, xs=xs)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, tem.default_options(tol=1e-13), keep_state=True)
    grad = res.state.adjoint(g)
    jd = res.state.jvp(dm)
    res.state.close()
    assert np.abs(grad - grad_ref).max() <= 1e-7 * np.abs(grad_ref).max()
    assert np.abs(jd - jd_ref).max() <= 1e-7 * np.abs(jd_ref).max()
