"""tem_forward_sources: several loops (the block source of Sec. 4) solved as one batch.

* the batched result equals separate tem_forward calls bit for bit (FP64 and mixed), since a
  system's arithmetic depends only on its own data;
* a loop with a current other than 1 A against the oracle (sparse LU), per-channel bound of
  the forward tests;
* bad input (a loop with two vertices, keep_state) is rejected before any launch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    m = W.uniform_model(16, 20.0, 5, 0.01, 60.0, 1e-5, 1e-3, 9, 10)
    _, xn = W._centres(m.hx, m.origin[0])
    _, yn = W._centres(m.hy, m.origin[1])
    loops = [W._square_loop(60.0, xn, yn),
             np.array([[xn[4], yn[5]], [xn[9], yn[5]], [xn[9], yn[8]], [xn[4], yn[8]]]),
             np.array([[xn[8], yn[8]], [xn[12], yn[8]], [xn[12], yn[13]], [xn[8], yn[13]]])]
    currents = np.array([1.0, 2.5, -0.7])
    rx = np.array([[0.0, 0.0, 0.0], [xn[10], yn[6], 0.0]])
    shifts, c, _ = R.tem_poles_residues(m.t, m.degree)
    return m, loops, currents, rx, shifts, c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_sources_equal_separate_forwards_bitwise(setup, prec):
    from paper_2506_11657_gb300 import tem
    m, loops, currents, rx, shifts, c = setup
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    opt = tem.default_options(precision=prec)
    D = tem.forward_sources(grid, loops, 0.0, rx, shifts, c, opt, currents=currents)
    assert D.shape == (3, 2, len(m.t))
    for j, (lp, cur) in enumerate(zip(loops, currents)):
        d = tem.forward(grid, lp, 0.0, rx, shifts, c, tem.default_options(precision=prec), current=cur).d
        assert np.array_equal(D[j], d), j


def test_scaled_current_matches_oracle(setup):
    from paper_2506_11657_gb300 import tem
    m, loops, currents, rx, shifts, c = setup
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, loops[1], 0.0, rx, current=currents[1], origin=m.origin)
    d, xs = P.forward(shifts, c, return_solutions=True)
    y = np.stack([P.Q @ x for x in xs])
    S = np.einsum("ik,ir->rk", np.abs(c), np.abs(y))
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    D = tem.forward_sources(grid, loops, 0.0, rx, shifts, c, tem.default_options(tol=1e-13), currents=currents)
    worst = np.max(np.abs(D[1] - d) / (1e-6 * np.abs(d) + 1e-10 * S))
    assert worst <= 1.0, worst


def test_sources_bad_input_rejected(setup):
    from paper_2506_11657_gb300 import tem
    m, loops, currents, rx, shifts, c = setup
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    n0 = tem.launch_count()
    with pytest.raises(tem.TEMError) as e:
        tem.forward_sources(grid, [loops[0], loops[1][:2]], 0.0, rx, shifts, c)
    assert e.value.code == tem.TEM_EINVAL
    with pytest.raises(tem.TEMError) as e:
        tem.forward_sources(grid, loops, 0.0, rx, shifts, c, tem.default_options(keep_state=1))
    assert e.value.code == tem.TEM_EINVAL
    assert tem.launch_count() == n0
