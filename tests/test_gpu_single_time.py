"""The single-time best-approximation baseline (Sec. 3.1, Eq. (rba)) through tem_forward_single_time:
one approximant of exp(-x) on [0, inf) evaluated at every channel on its own, i.e. the K * s
systems (t_k K - xi_i M) x = f.  Against the oracle's evaluation of the same systems (sparse LU,
shifts xi_i / t_k with the weights c_i / t_k on channel k), per channel to 1e-6; with degree 7
and K = 31 channels the count is the paper's 124 shifted solves (4 x 31), in two batches."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_single_time_baseline_matches_oracle():
    from paper_2506_11657_gb300 import tem
    from tests._parity import check, oracle_responses
    m = W.uniform_model(10, 20.0, 3, 0.01, 40.0, 1e-5, 1e-3, 31, 12)
    xi, c, _ = R.tem_poles_residues([1.0], 7)
    s, K = len(xi), len(m.t)
    shifts = np.array([xi[i] / tk for tk in m.t for i in range(s)])
    weights = np.zeros((s * K, K), dtype=np.complex128)
    for k, tk in enumerate(m.t):
        weights[k * s:(k + 1) * s, k] = c[:, 0] / tk
    (d_ref, S), = oracle_responses([(m, shifts, weights, None)])
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    d, solves = tem.forward_single_time(grid, m.loop_xy, m.z_loop, m.rx, m.t, xi, c[:, 0],
                                        tem.default_options(precision="fp64", tol=1e-13))
    grid.close()
    assert solves == 124 == K * s
    check(d, d_ref, S, 1e-6, 1e-10, "single-time baseline")
