"""Host logic of the Gauss-Newton / CGLS layer (no GPU): CGLS against a dense least-squares
solve, and one Gauss-Newton step on a linear stand-in for the forward (d(m) = A m), for which
one exact step must land on the damped least-squares minimiser — this pins the signs, the
Tikhonov extension, the data weights and the active-cell mask."""
import types

import numpy as np
import pytest

from paper_2506_11657_gb300 import inversion


def test_cgls_matches_dense_least_squares():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 15))
    b = rng.standard_normal(40)
    lam = 0.3
    Ae = np.vstack((A, np.sqrt(lam) * np.eye(15)))
    be = np.concatenate((b, np.zeros(15)))
    x, hist = inversion.cgls(lambda v: Ae @ v, lambda r: Ae.T @ r, be, 15)
    ref = np.linalg.lstsq(Ae, be, rcond=None)[0]
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()
    assert all(h1 <= h0 * (1 + 1e-12) for h0, h1 in zip(hist, hist[1:])), "CGLS residuals must not grow"


def test_cgls_zero_rhs():
    x, hist = inversion.cgls(lambda v: 2 * v, lambda r: 2 * r, np.zeros(5), 10)
    assert not np.any(x) and hist == [0.0]


class _FakeState:
    def __init__(self, A, shape):
        self.A, self.shape = A, shape

    def jvp(self, v):
        return (self.A @ v).reshape(self.shape)

    def adjoint(self, g):
        return self.A.T @ np.asarray(g).ravel()

    def close(self):
        pass


def test_gauss_newton_step_on_a_linear_forward(monkeypatch):
    rng = np.random.default_rng(1)
    n_rx, K, n = 2, 6, 9
    A = rng.standard_normal((n_rx * K, n))
    m_true = rng.standard_normal(n)
    d_obs = (A @ m_true).reshape(n_rx, K)
    active = np.ones(n, dtype=bool)
    active[[2, 7]] = False
    weights = 10 ** rng.uniform(-1, 1, (n_rx, K))
    lam = 0.05
    m0 = rng.standard_normal(n)
    m_ref = np.zeros(n)
    state = {}

    class Grid:
        def set_sigma(self, s):
            state["m"] = np.log(s)

    def forward(grid, loop_xy, z_loop, rx, shifts, c, options, keep_state=False):
        d = (A @ state["m"]).reshape(n_rx, K)
        return types.SimpleNamespace(d=d, status=0, state=_FakeState(A, (n_rx, K)))

    monkeypatch.setattr(inversion.tem, "forward", forward)
    model = types.SimpleNamespace(loop_xy=None, z_loop=0.0, rx=None)
    step = inversion.gauss_newton_step(Grid(), model, m0, d_obs, None, None, lam=lam, m_ref=m_ref,
                                       weights=weights, active=active, n_cgls=50)
    # the minimiser of ||W (A m - d_obs)||^2 + lam ||m - m_ref||^2 over the active cells
    W = weights.ravel()
    Aa = (W[:, None] * A)[:, active]
    rhs = W * (d_obs.ravel() - A[:, ~active] @ m0[~active])
    Ae = np.vstack((Aa, np.sqrt(lam) * np.eye(active.sum())))
    be = np.concatenate((rhs, np.sqrt(lam) * m_ref[active]))
    best = np.linalg.lstsq(Ae, be, rcond=None)[0]
    assert np.abs(step.m[active] - best).max() <= 1e-8 * np.abs(best).max()
    assert np.array_equal(step.m[~active], m0[~active])
    assert step.misfit == pytest.approx(np.linalg.norm(W * (A @ m0 - d_obs.ravel())))
