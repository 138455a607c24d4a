"""GPU field snapshots (tem_state_fields): the columns of S R in Sec. 3.2,
u_k = sum_i Re(c[i, k] x_i) on every edge.

* against the oracle's rational field from its LU solutions, per channel in the two norms of
  the problem: ||u - u_ref||_M and the curl energy ((u - u_ref)^T K (u - u_ref))^(1/2), each to
  1e-9 of sum_i |c[i, k]| times the same norm of x_i (FP64 solves to 1e-13).  Entry-wise the
  two differ in the air, where the curl-free part of the field is weakly determined
  (eigenvalue -xi sigma_air V of the gradient modes) and invisible to the response;
* against the exact exp(-t_k M^{-1} K) M^{-1} f (oracle T0, dense) within the M-norm bound of
  Sec. 3.3: ||u_exact - u_k||_M <= ||M^{-1} f||_M max_j |e^{-t_k lam_j} - r_k(lam_j)| over the
  spectrum lam_j of M^{-1} K (plus the solve error);
* a channel sub-range equals the same rows of the full call; bad ranges are rejected.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.solvers import DenseEig
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W
from tests._layout import lib_index_of_interior

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run():
    from paper_2506_11657_gb300 import tem
    m = W.uniform_model(10, 20.0, 3, 0.01, 40.0, 1e-5, 1e-3, 9, 10)
    shifts, c, _ = R.tem_poles_residues(m.t, m.degree)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, tem.default_options(tol=1e-13), keep_state=True)
    U = res.state.fields().cpu().numpy()
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    idx = lib_index_of_interior(P.grid)
    return tem, m, shifts, c, res, U, P, idx


def test_fields_match_the_oracle_rational_field(run):
    tem, m, shifts, c, res, U, P, idx = run
    d, xs = P.forward(shifts, c, return_solutions=True)
    X = np.stack(xs)                                     # (s, N) interior edges
    pad = np.ones(U.shape[1], dtype=bool)
    pad[idx] = False
    assert not np.any(U[:, pad])
    nM = np.sqrt((P.Md[None, :] * np.abs(X) ** 2).sum(axis=1))                  # ||x_i||_M
    nK = np.sqrt(np.abs(np.einsum("in,in->i", X.conj(), (P.K @ X.T).T)))          # |x_i^H K x_i|^(1/2)
    for k in range(len(m.t)):
        diff = U[k, idx] - (c[:, k][:, None] * X).real.sum(axis=0)
        errM = np.sqrt(np.sum(P.Md * diff * diff))
        errK = np.sqrt(abs(diff @ (P.K @ diff)))
        assert errM <= 1e-9 * np.sum(np.abs(c[:, k]) * nM), (k, errM)
        assert errK <= 1e-9 * np.sum(np.abs(c[:, k]) * nK), (k, errK)


def test_fields_within_the_m_norm_bound_of_the_exact_field(run):
    tem, m, shifts, c, res, U, P, idx = run
    E = DenseEig(P.K, P.Md)
    b = P.f / P.Md
    bM = np.sqrt(np.sum(P.Md * b * b))
    for k, tk in enumerate(m.t):
        exact = E.expm(tk, P.f)
        r = sum((ci / (E.lam - xi)).real for xi, ci in zip(shifts, c[:, k]))
        eps = np.abs(np.exp(-tk * E.lam) - r).max()
        diff = exact - U[k, idx]
        errM = np.sqrt(np.sum(P.Md * diff * diff))
        assert errM <= 1.01 * bM * eps + 1e-9 * bM, (k, errM, bM * eps)


def test_fields_subrange_and_invalid(run):
    tem, m, shifts, c, res, U, P, idx = run
    part = res.state.fields(3, 2).cpu().numpy()
    assert np.array_equal(part, U[3:5])
    for k0, nk in [(-1, 1), (0, 0), (len(m.t) - 1, 2)]:
        out = torch.empty((2, 3 * res.state.n_cells), dtype=torch.float64, device="cuda")
        with pytest.raises(tem.TEMError) as e:
            res.state.fields(k0, nk, out=out)
        assert e.value.code == tem.TEM_EINVAL
