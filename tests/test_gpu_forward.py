"""GPU parity of tem_forward (FP64 and mixed precision) against the oracle, plus failure paths.

Parity is defined for fixed shifts and channel weights (both sides consume the same
(xi, c)): d[r, k] = sum_i Re(c[i, k] q_r^T (K - xi_i M)^{-1} f).  Every channel must meet the
plain relative error |d_gpu - d_oracle| <= rel |d_oracle|: rel = 1e-6 for FP64 (solves to an
FP64 residual of 1e-13), rel = 1e-5 for mixed precision (FP32 sweeps, FP64 residual 1e-12).
The check also prints the ratio to rel |d| + floor S_k, S_k = sum_i |c[i, k] y_i| (the size of
the pole terms before they cancel), as a diagnostic of how close a channel is to the
cancellation limit of FP64 arithmetic.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle(m, shifts, c, rx=None):
    rx = m.rx if rx is None else rx
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    d, xs = P.forward(shifts, c, return_solutions=True)
    y = np.stack([P.Q @ x for x in xs])            # (s, n_rx)
    S = np.einsum("ik,ir->rk", np.abs(c), np.abs(y))
    return d, S


def _check(d_gpu, d_ref, S, rel, floor):
    from tests._parity import check
    return check(d_gpu, d_ref, S, rel, floor, f"forward (rel {rel:g}, floor {floor:g})")


@pytest.fixture(scope="module")
def tiny():
    m = W.tiny16()
    shifts, c, _ = R.tem_poles_residues(m.t, m.degree)
    rx = np.array([[0.0, 0.0, 0.0], [25.0, -13.0, 0.0], [-70.0, 55.0, 0.0]])
    d_ref, S = _oracle(m, shifts, c, rx)
    return m, shifts, c, rx, d_ref, S


def test_tiny16_fp64_matches_oracle(tiny):
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d_ref, S = tiny
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, tem.default_options(tol=1e-13))
    assert res.status == tem.TEM_OK
    _check(res.d, d_ref, S, 1e-6, 1e-10)


@pytest.mark.parametrize("carry", [0, 1])
@pytest.mark.parametrize("precond", ["nodal", "jacobi"])
def test_tiny16_mixed_matches_oracle(tiny, precond, carry):
    """Both outer schemes: restart every inner solve (carry 0) and residual replacement with
    the search direction kept across outer steps (carry 1)."""
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d_ref, S = tiny
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    opt = tem.default_options(precision="mixed", tol=1e-12, precond=precond, inner_tol=1e-3 if precond == "nodal" else 1e-1,
                              carry_direction=carry)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt)
    assert res.status == tem.TEM_OK
    _check(res.d, d_ref, S, 1e-5, 1e-9)


@pytest.mark.parametrize("precond", ["jacobi", "nodal"])
@pytest.mark.parametrize("dims", [(34, 10, 12), (20, 18, 40)])
def test_ragged_grids_fp64(dims, precond):
    """Tiles of 32 x 8 nodes and 32-plane chunks with ragged tails in x, y and z; both
    preconditioners (they change the iterates, not the solution)."""
    from paper_2506_11657_gb300 import tem
    nx, ny, nz = dims
    m = W.uniform_model(nx, 10.0, nz // 3, 0.02, 60.0, 1e-5, 1e-3, 9, 8, ny=ny, nz=nz)
    shifts, c, _ = R.tem_poles_residues(m.t, m.degree)
    rx = np.array([[0.0, 0.0, 0.0], [12.0, 7.0, 0.0]])
    d_ref, S = _oracle(m, shifts, c, rx)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, tem.default_options(tol=1e-13, precond=precond))
    _check(res.d, d_ref, S, 1e-6, 1e-10)


def test_deterministic_and_conjugate_invariant(tiny):
    """Same call twice: bitwise equal.  Conjugated shifts and weights: same response
    (Re(conj(c) conj(y)) = Re(c y) since K, M, f, q are real)."""
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d_ref, S = tiny
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    opt = tem.default_options(tol=1e-13)
    a = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
    b = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt).d
    assert np.array_equal(a, b)
    cc = tem.forward(grid, m.loop_xy, m.z_loop, rx, np.conj(shifts), np.conj(c), opt).d
    _check(cc, d_ref, S, 1e-6, 1e-10)


def test_enoconv_still_writes_output(tiny):
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d_ref, S = tiny
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, tem.default_options(max_iter=3, max_outer=2))
    assert res.status == tem.TEM_ENOCONV
    assert np.all(np.isfinite(res.d))


def test_invalid_inputs_rejected(tiny):
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d_ref, S = tiny
    bad = m.sigma.copy()
    bad.flat[5] = np.nan
    with pytest.raises(tem.TEMError) as e:
        tem.Grid(m.hx, m.hy, m.hz, m.origin, bad)
    assert e.value.code == tem.TEM_EINVAL
    bad.flat[5] = -1.0
    with pytest.raises(tem.TEMError):
        tem.Grid(m.hx, m.hy, m.hz, m.origin, bad)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    with pytest.raises(tem.TEMError) as e:  # loop vertex off the node grid
        tem.forward(grid, m.loop_xy + 3.0, m.z_loop, rx, shifts, c)
    assert e.value.code == tem.TEM_EINVAL
    with pytest.raises(tem.TEMError):  # receiver outside the grid
        tem.forward(grid, m.loop_xy, m.z_loop, np.array([[1e5, 0.0, 0.0]]), shifts, c)
    with pytest.raises(tem.TEMError):  # a real shift on the spectrum
        tem.forward(grid, m.loop_xy, m.z_loop, rx, np.array([5.0 + 0j]), c[:1])
