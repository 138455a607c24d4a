"""The adjoint gradient on the 96^3 model (Sec. 4): 64 surface receivers of d_t b_z at 31
channels, 20 poles, a layered 300 Ohm m host with four conductive blocks.

The misfit is phi = 1/2 sum_{r,k} ((d_rk - d_obs,rk) / |d_obs,rk|)^2 with d_obs the response of the
layered background (the blocks removed), so dphi/dd = (d - d_obs) / d_obs^2.

* 96^3: the gradient from tem_adjoint against central differences of the forward (delta = 1e-3
  in log sigma, solves to an FP64 residual of 1e-13) on 32 seeded earth cells within 200 m of the
  loop centre, accepted within 1e-4 of max |g|.
* 24^3 with 40 m cells (the same physical model, 4x coarser): J^T g for a seeded g, FP64, against
  the oracle's (sparse LU for the forward and adjoint solves) on every cell, within 1e-7 of the
  largest entry.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _misfit(d, d_obs):
    r = (d - d_obs) / np.abs(d_obs)
    return 0.5 * float(np.sum(r * r)), (d - d_obs) / d_obs ** 2


def test_adjoint96_gradient_matches_finite_differences():
    from paper_2506_11657_gb300 import tem
    m = W.adjoint96()
    bg = W.adjoint96(blocks=False)
    shifts, c, _ = tem.poles_residues(m.t, m.degree)
    opt = tem.default_options(precision="mixed", tol=1e-13)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, bg.sigma)
    d_obs = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, opt).d
    grid.set_sigma(m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, opt, keep_state=True)
    assert res.status == tem.TEM_OK
    phi0, g_d = _misfit(res.d, d_obs)
    assert phi0 > 0
    grad = res.state.adjoint(g_d)
    res.state.close()
    # 32 seeded earth cells whose centres lie within 200 m of the loop centre
    n = len(m.hx)
    xc = m.origin[0] + np.cumsum(m.hx) - 0.5 * m.hx
    zc = m.origin[2] + np.cumsum(m.hz) - 0.5 * m.hz
    lc = m.loop_xy.mean(axis=0)
    Z, Y, X = np.meshgrid(zc, xc, xc, indexing="ij")
    near = (np.sqrt((X - lc[0]) ** 2 + (Y - lc[1]) ** 2 + Z ** 2) <= 200.0) & (m.sigma > 1e-6)
    cand = np.flatnonzero(near.ravel())
    cells = np.random.default_rng(32).choice(cand, size=32, replace=False)
    delta = 1e-3
    logs = np.log(m.sigma.ravel())
    fd = []
    for cell in cells:
        phis = []
        for sgn in (1, -1):
            ls = logs.copy()
            ls[cell] += sgn * delta
            grid.set_sigma(np.exp(ls).reshape(m.sigma.shape))
            r = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, opt)
            assert r.status == tem.TEM_OK
            phis.append(_misfit(r.d, d_obs)[0])
        fd.append((phis[0] - phis[1]) / (2 * delta))
    grid.close()
    fd = np.array(fd)
    scale = np.abs(grad).max()
    err = np.abs(fd - grad[cells]) / scale
    print(f"adjoint96: max |g| {scale:.3e}, max |g_fd - g_adj| / max|g| over 32 cells {err.max():.2e}")
    assert err.max() <= 1e-4, err.max()


def test_adjoint96_coarse_gradient_matches_oracle():
    """J^T g on the 4x coarsening (24^3 cells of 40 m, the same 64 receivers, 20 poles) for a
    seeded g: tem_adjoint (FP64 solves to 1e-13) against the oracle's sparse-LU adjoint on every
    cell, within 1e-7 of max |g|."""
    from paper_2506_11657_gb300 import tem
    from tests._parity import oracle_adjoint
    m = W.adjoint96(n=24, h=40.0)
    shifts, c, _ = tem.poles_residues(m.t, m.degree)
    g = np.random.default_rng(24).standard_normal((len(m.rx), len(m.t)))
    grad_ref = oracle_adjoint(m, shifts, c, g)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, tem.default_options(precision="fp64", tol=1e-13),
                      keep_state=True)
    grad = res.state.adjoint(g)
    res.state.close()
    grid.close()
    scale = np.abs(grad_ref).max()
    err = np.abs(grad - grad_ref.ravel()) / scale
    print(f"adjoint96 coarse 24^3: J^T g max err / max|J^T g| {err.max():.2e}")
    assert err.max() <= 1e-7, err.max()
