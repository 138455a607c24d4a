"""Gauss-Newton (Sec. 4) through the GPU J and J^T actions: from the background model towards
a model with a conductive block, data weighted by a 5 % relative error with a floor, the update
on the earth cells only.  The damped linear problem must shrink under CGLS, and two
backtracking Gauss-Newton iterations must lower the objective monotonically, by more than 30 %."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_gauss_newton_step_reduces_the_misfit():
    from paper_2506_11657_gb300 import inversion, tem
    m = W.uniform_model(16, 10.0, 5, 0.01, 60.0, 1e-5, 1e-2, 10, 12, ny=14, nz=18)
    background = m.sigma.copy()
    true = background.copy()
    true[9:13, 5:9, 6:10] *= 5.0          # a conductive block below the loop (z, y, x cells)
    rx = np.array([[0.0, 0.0, 0.0], [20.0, 10.0, 0.0], [-20.0, -10.0, 0.0], [30.0, -20.0, 0.0]])
    m.rx = rx
    shifts, c, _ = tem.poles_residues(m.t, 12)
    opt = tem.default_options(tol=1e-12)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, true)
    d_obs = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
    weights = 1.0 / (0.05 * np.abs(d_obs) + 1e-3 * np.abs(d_obs).max())
    active = (background > 1e-6).ravel()
    m0 = np.log(background.ravel())
    step = inversion.gauss_newton_step(grid, m, m0, d_obs, shifts, c, opt, lam=1e-4, weights=weights,
                                       active=active, n_cgls=6)
    assert np.all(np.isfinite(step.m))
    assert np.array_equal(step.m[~active], m0[~active])
    assert step.cgls_residuals[-1] < 0.5 * step.cgls_residuals[0]
    m2, hist = inversion.gauss_newton(grid, m, m0, d_obs, shifts, c, opt, n_steps=2, lam=1e-4, weights=weights,
                                      active=active, n_cgls=6)
    print("gauss-newton objective", hist)
    assert len(hist) == 3 and hist[2] < hist[1] < hist[0], hist
    assert hist[2] < 0.7 * hist[0], hist
    assert np.array_equal(m2[~active], m0[~active])
