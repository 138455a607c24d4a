"""Limits and degenerate cases of tem_forward against the oracle (sparse LU per shift):

* the largest batch the entry point takes: 64 shifts (complex ones in both half-planes and
  real negative ones), 64 receivers, 9 channels with random complex weights, FP64 and mixed;
* the smallest: one real pole (degree 1), one channel, one receiver;
* one past each limit (65 shifts, 4097 receivers) is rejected before any device work.

Parity is the plain per-channel relative error of the forward tests,
|d_gpu - d_oracle| <= rel |d_oracle| (FP64 1e-6, mixed 1e-5).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rational as R
from oracle.tem import TEMProblem
from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _oracle(m, shifts, c, rx):
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, rx, origin=m.origin)
    d, xs = P.forward(shifts, c, return_solutions=True)
    y = np.stack([P.Q @ x for x in xs])
    return d, np.einsum("ik,ir->rk", np.abs(c), np.abs(y))


def _check(d, ref, S, rel, floor):
    from tests._parity import check
    return check(d, ref, S, rel, floor, f"limits (rel {rel:g}, floor {floor:g})")


@pytest.fixture(scope="module")
def big_batch():
    m = W.uniform_model(12, 20.0, 3, 0.02, 60.0, 1e-5, 1e-3, 9, 10, ny=11, nz=13)
    rng = np.random.default_rng(41)
    # 64 shifts off [0, inf): complex in the left and right half-planes, and real negative ones
    mag = 10 ** rng.uniform(3.0, 6.0, 64)
    ang = rng.uniform(0.15 * np.pi, 0.95 * np.pi, 64)
    shifts = mag * np.exp(1j * ang)
    shifts[:6] = -mag[:6]
    c = (rng.standard_normal((64, 9)) + 1j * rng.standard_normal((64, 9))) * mag[:, None] * 1e-6
    xs = np.linspace(-90.0, 90.0, 8)
    rx = np.array([[x, y, 0.0] for x in xs for y in np.linspace(-80.0, 80.0, 8)])
    d, S = _oracle(m, shifts, c, rx)
    return m, shifts, c, rx, d, S


@pytest.mark.parametrize("prec,rel,floor", [("fp64", 1e-6, 1e-10), ("mixed", 1e-5, 1e-9)])
def test_64_shifts_64_receivers(big_batch, prec, rel, floor):
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d, S = big_batch
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    opt = tem.default_options(precision=prec, tol=1e-13 if prec == "fp64" else 1e-12)
    res = tem.forward(grid, m.loop_xy, m.z_loop, rx, shifts, c, opt)
    assert res.status == tem.TEM_OK
    assert res.d.shape == (64, 9)
    _check(res.d, d, S, rel, floor)


def test_one_real_pole_one_channel_one_receiver():
    from paper_2506_11657_gb300 import tem
    m = W.uniform_model(10, 20.0, 3, 0.01, 40.0, 1e-4, 1e-4, 1, 1)
    shifts, c, err = tem.poles_residues(m.t, 1)
    assert shifts.shape == (1,) and shifts[0].imag == 0.0 and shifts[0].real < 0.0
    d, S = _oracle(m, shifts, c, m.rx)
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    res = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, shifts, c, tem.default_options(tol=1e-13))
    assert res.status == tem.TEM_OK and res.d.shape == (1, 1)
    _check(res.d, d, S, 1e-6, 1e-10)


def test_one_past_each_limit_is_rejected(big_batch):
    from paper_2506_11657_gb300 import tem
    m, shifts, c, rx, d, S = big_batch
    grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    n0 = tem.launch_count()
    s65 = np.concatenate((shifts, shifts[:1]))
    c65 = np.concatenate((c, c[:1]))
    with pytest.raises(tem.TEMError) as e:
        tem.forward(grid, m.loop_xy, m.z_loop, rx, s65, c65)
    assert e.value.code == tem.TEM_EINVAL
    rx_many = np.zeros((4097, 3))
    with pytest.raises(tem.TEMError) as e:
        tem.forward(grid, m.loop_xy, m.z_loop, rx_many, shifts[:2], c[:2])
    assert e.value.code == tem.TEM_EINVAL
    assert tem.launch_count() == n0, "rejected calls launch nothing"
