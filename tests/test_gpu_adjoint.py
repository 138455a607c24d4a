"""GPU parity of tem_adjoint (Sec. 4) against the oracle's adjoint, finite differences of the GPU
forward, and the torch.autograd wrapper.

The gradient of phi = sum(g * d) w.r.t. log sigma is
    dphi/dlog sigma_c = sum_i Re( xi_i lambda_i^T (sigma_c V_c / 4 on the cell's edges) x_i ),
lambda_i = (K - xi_i M)^{-1} sum_r beta[i, r] q_r,  beta = c g^T.  It is compared per cell
against the oracle (sparse LU for both the forward and the adjoint solves) relative to the
largest gradient entry: 1e-7 for FP64 solves to 1e-13, 1e-5 for mixed precision.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    # a small ragged grid with a layered, blocky earth (conductive blocks in a resistive host)
    m = W.uniform_model(16, 10.0, 5, 1.0 / 300.0, 60.0, 1e-5, 1e-2, 10, 12, ny=14, nz=18)
    rng = np.random.default_rng(21)
    s = m.sigma.copy()
    earth = s > 1e-6
    s[earth] *= 10 ** rng.uniform(-0.5, 1.2, earth.sum())
    m.sigma = s
    rx = np.array([[0.0, 0.0, 0.0], [15.0, 5.0, 0.0], [-25.0, 12.0, 0.0], [35.0, -30.0, 0.0],
                   [5.0, 40.0, 0.0], [-40.0, -20.0, 0.0]])
    t = m.t
    shifts, c, _ = R.tem_poles_residues(t, 12)
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    d, xs = P.forward(shifts, c, return_solutions=True)
    g = rng.standard_normal(d.shape) / np.abs(d).mean()
    grad = P.adjoint_gradient(shifts, c, g, xs=xs)
    return m, rx, shifts, c, d, g, grad


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("mixed", 1e-5)])
def test_adjoint_matches_oracle(problem, prec, tol):
    from paper_2506_11657_gb300 import tem
    m, rx, shifts, c, d, g, grad = problem
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    opt = tem.default_options(precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt, keep_state=True)
    ga = res.state.adjoint(g)
    res.state.close()
    scale = np.abs(grad).max()
    err = np.abs(ga - grad).max() / scale
    assert err <= tol, err
    # air cells carry (almost) no sensitivity; the earth cells near the loop carry most
    assert np.abs(ga).argmax() == np.abs(grad).argmax()


def test_adjoint_matches_gpu_finite_differences(problem):
    """Central differences of the GPU forward in log sigma on a few cells."""
    from paper_2506_11657_gb300 import tem
    m, rx, shifts, c, d, g, grad = problem
    opt = tem.default_options(tol=1e-13)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt, keep_state=True)
    ga = res.state.adjoint(g)
    res.state.close()
    order = np.argsort(-np.abs(ga))
    cells = list(order[:4]) + list(np.random.default_rng(3).choice(order[:200], 3, replace=False))
    h = 1e-4
    for cell in cells:
        sp, sm = m.sigma.ravel().copy(), m.sigma.ravel().copy()
        sp[cell] *= np.exp(h)
        sm[cell] *= np.exp(-h)
        grid.set_sigma(sp)
        dp = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
        grid.set_sigma(sm)
        dm = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
        fd = ((dp - dm) * g).sum() / (2 * h)
        assert abs(fd - ga[cell]) <= 1e-5 * np.abs(ga).max(), (cell, fd, ga[cell])


def test_autograd_function_backward(problem):
    from paper_2506_11657_gb300 import tem
    from paper_2506_11657_gb300.autograd import tem_forward_logsigma
    m, rx, shifts, c, d, g, grad = problem
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    ls = torch.tensor(np.log(m.sigma.ravel()), dtype=torch.float64, requires_grad=True)
    out = tem_forward_logsigma(ls, grid, m.loop_xy, m.z_loop, rx, shifts, c, tem.default_options(tol=1e-13))
    assert np.allclose(out.detach().numpy(), d, rtol=1e-6, atol=1e-10 * np.abs(d).max())
    (out * torch.from_numpy(g)).sum().backward()
    assert np.abs(ls.grad.numpy() - grad).max() <= 1e-7 * np.abs(grad).max()


def test_stale_state_is_refused_and_autograd_recovers(problem):
    """A kept state belongs to the conductivity of its forward call: after tem_grid_set_sigma the
    library refuses tem_adjoint and tem_jvp on it, and the autograd wrapper, given two forwards on
    one grid before either backward, still returns both gradients."""
    from paper_2506_11657_gb300 import tem
    from paper_2506_11657_gb300.autograd import tem_forward_logsigma
    m, rx, shifts, c, d, g, grad = problem
    opt = tem.default_options(tol=1e-13)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt, keep_state=True)
    grid.set_sigma(m.sigma * 1.5)
    for call in (lambda: res.state.adjoint(g), lambda: res.state.jvp(np.ones(m.sigma.size))):
        with pytest.raises(tem.TEMError) as e:
            call()
        assert e.value.code == tem.TEM_EINVAL
    res.state.close()
    ls1 = torch.tensor(np.log(m.sigma.ravel()), dtype=torch.float64, requires_grad=True)
    ls2 = torch.tensor(np.log(m.sigma.ravel() * 1.5), dtype=torch.float64, requires_grad=True)
    o1 = tem_forward_logsigma(ls1, grid, m.loop_xy, m.z_loop, rx, shifts, c, opt)
    o2 = tem_forward_logsigma(ls2, grid, m.loop_xy, m.z_loop, rx, shifts, c, opt)
    gt = torch.from_numpy(g)
    ((o1 * gt).sum() + (o2 * gt).sum()).backward()
    assert np.abs(ls1.grad.numpy() - grad).max() <= 1e-7 * np.abs(grad).max()
    grid.set_sigma(m.sigma * 1.5)
    r2 = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt, keep_state=True)
    g2 = r2.state.adjoint(g)
    r2.state.close()
    assert np.abs(ls2.grad.numpy() - g2).max() <= 1e-9 * np.abs(g2).max()
    grid.close()
