"""GPU parity of tem_jvp, the linearised forward of Sec. 4 (J dm for a direction dm in log sigma).

    dd[r, k] = sum_i Re(c[i, k] q_r^T dx_i),   dx_i = (K - xi_i M)^{-1} (xi_i dM x_i),
    dM = diag(sum_c dm_c sigma_c M_c).

Checked against the oracle's J dm (sparse LU for the forward and the linearised solves) with
the plain per-channel relative error of the forward tests, |dd_gpu - dd_oracle| <= rel |dd_oracle|
(FP64 solves to 1e-13: rel 1e-6; mixed: 1e-5), against central differences of the GPU forward,
and against tem_adjoint through <g, J dm> = <J^T g, dm>.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.solvers import solve_lu
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    m = W.uniform_model(16, 10.0, 5, 1.0 / 300.0, 60.0, 1e-5, 1e-2, 10, 12, ny=14, nz=18)
    rng = np.random.default_rng(31)
    s = m.sigma.copy()
    earth = s > 1e-6
    s[earth] *= 10 ** rng.uniform(-0.5, 1.2, earth.sum())
    m.sigma = s
    rx = np.array([[0.0, 0.0, 0.0], [15.0, 5.0, 0.0], [-25.0, 12.0, 0.0], [35.0, -30.0, 0.0]])
    shifts, c, _ = R.tem_poles_residues(m.t, 12)
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    d, xs = P.forward(shifts, c, return_solutions=True)
    dm = rng.standard_normal(m.sigma.size) * earth.ravel()   # perturb the earth cells
    jd = P.jvp(shifts, c, dm, xs=xs)
    # S'_k from the oracle's linearised solutions
    dM = P.mass_derivative() @ dm
    y = np.stack([P.Q @ solve_lu(P.K, P.Md, sh * (dM * xs[i]), sh) for i, sh in enumerate(shifts)])
    S = np.einsum("ik,ir->rk", np.abs(c), np.abs(y))
    return m, rx, shifts, c, dm, jd, S, rng


def _check(dd, ref, S, rel, floor):
    from tests._parity import check
    return check(dd, ref, S, rel, floor, f"J dm (rel {rel:g}, floor {floor:g})")


@pytest.mark.parametrize("prec,rel,floor", [("fp64", 1e-6, 1e-10), ("mixed", 1e-5, 1e-9)])
@pytest.mark.parametrize("precond", ["nodal", "jacobi"])
def test_jvp_matches_oracle(problem, prec, rel, floor, precond):
    from paper_2506_11657_gb300 import tem
    m, rx, shifts, c, dm, jd, S, rng = problem
    if prec == "mixed" and precond == "jacobi":
        opt = tem.default_options(precision=prec, precond=precond, inner_tol=1e-1)
    else:
        opt = tem.default_options(precision=prec, precond=precond, tol=1e-13 if prec == "fp64" else 1e-12)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt, keep_state=True)
    dd = res.state.jvp(dm)
    res.state.close()
    _check(dd, jd, S, rel, floor)


def test_jvp_is_the_transpose_of_the_gpu_adjoint(problem):
    from paper_2506_11657_gb300 import tem
    m, rx, shifts, c, dm, jd, S, rng = problem
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, tem.default_options(tol=1e-13), keep_state=True)
    g = rng.standard_normal(res.d.shape)
    dd = res.state.jvp(dm)
    gr = res.state.adjoint(g)
    res.state.close()
    lhs, rhs = np.sum(g * dd), np.dot(gr, dm)
    assert abs(lhs - rhs) <= 1e-8 * (np.sum(np.abs(g * dd)) + np.sum(np.abs(gr * dm))), (lhs, rhs)


def test_jvp_matches_gpu_finite_differences(problem):
    from paper_2506_11657_gb300 import tem
    m, rx, shifts, c, dm, jd, S, rng = problem
    opt = tem.default_options(tol=1e-13)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt, keep_state=True)
    dd = res.state.jvp(dm)
    res.state.close()
    h = 1e-4
    grid.set_sigma(m.sigma.ravel() * np.exp(h * dm))
    dp = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
    grid.set_sigma(m.sigma.ravel() * np.exp(-h * dm))
    dn = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
    fd = (dp - dn) / (2 * h)
    assert np.abs(fd - dd).max() <= 1e-5 * np.abs(dd).max()


def test_jvp_degenerate_and_invalid(problem):
    from paper_2506_11657_gb300 import tem
    m, rx, shifts, c, dm, jd, S, rng = problem
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, tem.default_options(), keep_state=True)
    n0 = tem.launch_count()
    assert not np.any(res.state.jvp(np.zeros(m.sigma.size)))
    assert tem.launch_count() == n0, "a zero direction needs no solve"
    bad = dm.copy()
    bad[5] = np.nan
    with pytest.raises(tem.TEMError) as e:
        res.state.jvp(bad)
    assert e.value.code == tem.TEM_EINVAL
    with pytest.raises(ValueError):
        res.state.jvp(dm[:-1])
    res.state.close()
