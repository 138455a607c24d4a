"""Host logic without a GPU: the autograd wrapper, the request-stream driver and its pole
cache (each against a stand-in for the library), and the seeded workloads the benchmark and
its stored iteration counts depend on."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W


def _standin(monkeypatch, A):
    """A linear stand-in d = A log sigma whose kept state, like the library's, refuses an adjoint
    once the grid's conductivity has changed after its forward call."""
    from paper_2506_11657_gb300 import autograd
    calls = {"forward": 0, "closed": 0}

    class Grid:
        def set_sigma(self, s):
            self.ls = np.log(s)

    class State:
        def __init__(self, grid):
            self.grid, self.ls = grid, grid.ls.copy()

        def adjoint(self, g):
            if not np.array_equal(self.grid.ls, self.ls):
                raise autograd.tem.TEMError(autograd.tem.TEM_EINVAL, "tem_adjoint")
            return A.T @ np.asarray(g).ravel()

        def close(self):
            calls["closed"] += 1

    def forward(g, loop_xy, z_loop, rx, shifts, c, options, keep_state=False):
        assert keep_state
        calls["forward"] += 1
        return types.SimpleNamespace(d=(A @ g.ls).reshape(2, 5), status=0, state=State(g))

    monkeypatch.setattr(autograd.tem, "forward", forward)
    monkeypatch.setattr(autograd.tem, "last_error", lambda: "")
    monkeypatch.setattr(autograd.tem, "status_string", lambda code: "EINVAL")
    return autograd, Grid(), calls


def test_autograd_backward_is_the_adjoint(monkeypatch):
    """With a linear stand-in d = A log sigma, backward must return A^T g, twice if asked."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((2 * 5, 12))
    autograd, grid, calls = _standin(monkeypatch, A)
    ls = torch.tensor(rng.standard_normal(12), dtype=torch.float64, requires_grad=True)
    d = autograd.TEMForward.apply(ls, grid, None, 0.0, None, None, None, None)
    assert np.allclose(d.detach().numpy(), (A @ ls.detach().numpy()).reshape(2, 5))
    g = torch.tensor(rng.standard_normal((2, 5)), dtype=torch.float64)
    (d * g).sum().backward(retain_graph=True)
    assert np.allclose(ls.grad.numpy(), A.T @ g.numpy().ravel())
    (d * g).sum().backward()
    assert np.allclose(ls.grad.numpy(), 2 * A.T @ g.numpy().ravel())
    assert calls["forward"] == 1


def test_autograd_two_forwards_on_one_grid(monkeypatch):
    """Two forwards on one grid before either backward: the first backward finds its state
    stale, sets its own conductivity again and repeats the forward; both gradients are right."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((2 * 5, 12))
    autograd, grid, calls = _standin(monkeypatch, A)
    l1 = torch.tensor(rng.standard_normal(12), dtype=torch.float64, requires_grad=True)
    l2 = torch.tensor(rng.standard_normal(12), dtype=torch.float64, requires_grad=True)
    d1 = autograd.TEMForward.apply(l1, grid, None, 0.0, None, None, None, None)
    d2 = autograd.TEMForward.apply(l2, grid, None, 0.0, None, None, None, None)
    g1 = torch.tensor(rng.standard_normal((2, 5)), dtype=torch.float64)
    g2 = torch.tensor(rng.standard_normal((2, 5)), dtype=torch.float64)
    ((d1 * g1).sum() + (d2 * g2).sum()).backward()
    assert np.allclose(l1.grad.numpy(), A.T @ g1.numpy().ravel())
    assert np.allclose(l2.grad.numpy(), A.T @ g2.numpy().ravel())
    assert calls["forward"] == 3 and calls["closed"] == 1


class _FakeServer:
    """Finishes each request `steps_needed` steps after its submission."""

    def __init__(self, steps_needed, clock):
        self.need, self.clock = steps_needed, clock
        self.jobs, self.nstep = {}, 0

    def submit(self, model, sh, c):
        tk = len(self.jobs)
        self.jobs[tk] = [self.nstep + self.need, self.clock(), model]
        return tk

    def step(self):
        self.nstep += 1
        self.clock.advance(0.1)

    def poll(self, tk):
        done_at, sub, model = self.jobs[tk]
        if self.nstep < done_at:
            return None
        return np.full((1, 3), float(tk)), {"admit_s": sub, "submit_s": sub, "status": 0}


class _Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def advance(self, dt):
        self.t += dt


def test_run_stream_latency_and_order(monkeypatch):
    from paper_2506_11657_gb300 import serving
    calls = []
    monkeypatch.setattr(serving.tem, "poles_residues", lambda t, m: calls.append((tuple(t), m)) or (None, None, 0.0))
    clock = _Clock()
    srv = _FakeServer(3, clock)
    m = W.uniform_model(4, 10.0, 1, 0.01, 20.0, 1e-5, 1e-3, 3, 4)
    items = [(0.25, m), (0.0, m), (0.55, m)]               # out of arrival order on purpose
    res, summ = serving.run_stream(srv, items, clock=clock, sleep=clock.advance)
    assert summ["requests"] == 3 and summ["failed"] == 0
    assert len(calls) == 1, "one fit per (times, degree)"
    for q, r in enumerate(res):
        assert r["arrival_s"] == items[q][0]
        assert r["done_s"] >= r["arrival_s"]
        assert r["latency_s"] == pytest.approx(r["done_s"] - r["arrival_s"])
    # the request arriving first is submitted first (ticket 0)
    assert res[1]["d"][0, 0] == 0.0
    with pytest.raises(RuntimeError):
        serving.run_stream(_FakeServer(10 ** 9, _Clock()), [(0.0, m)], clock=_Clock(), sleep=lambda s: None,
                           max_wall_s=-1.0)


def test_bench_workload_is_pinned():
    """The 128^3 benchmark model (the stored iteration counts and bench lines refer to it)."""
    m = W.randblock128()
    assert m.sigma.shape == (128, 128, 128) and m.degree == 20 and len(m.t) == 31
    assert m.origin == (-640.0, -640.0, -1120.0)
    assert np.array_equal(m.loop_xy, [[-100.0, -100.0], [100.0, -100.0], [100.0, 100.0], [-100.0, 100.0]])
    assert np.array_equal(m.rx, [[0.0, 0.0, 0.0]])
    assert np.isclose(m.t[0], 1e-5, rtol=1e-14) and np.isclose(m.t[-1], 1e-2, rtol=1e-14)
    s = m.sigma
    assert np.isclose(s.sum(), 279512.87079729873, rtol=1e-12)
    assert np.isclose(np.log10(s).mean(), -2.2993018088349184, rtol=1e-12)
    assert np.isclose(s[50, 60, 70], 0.28424578959525265, rtol=1e-12)
    assert np.isclose(s[3, 100, 7], 0.002348049730594285, rtol=1e-12)
    assert np.all(s[128 - 16:] == W.SIGMA_AIR)


def test_serving_stream_is_pinned():
    items = W.serving_stream(n_requests=8, seed=4)
    assert [m.shape for _, m in items] == [(64,) * 3, (48,) * 3, (48,) * 3, (96,) * 3, (32,) * 3, (32,) * 3,
                                           (48,) * 3, (48,) * 3]
    assert [m.degree for _, m in items] == [20, 18, 20, 19, 18, 20, 20, 17]
    assert np.allclose([a for a, _ in items], [3.798827, 4.229625, 7.469825, 7.611016, 8.551266, 9.34634,
                                               9.960733, 11.478622], atol=1e-6)


def test_bench_byte_counts():
    """The bytes per interior edge per shift that the bench divides by each pass's time, tallied
    here array by array (complex FP32 = 8 B per entry; a nodal vector has one entry per three
    edges; per-grid arrays are shared by the s shifts that sweep a tile together)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    s = 10
    node = 8.0 / 3.0
    pb = bench.pass_bytes(s)
    # two-pass COCG without a preconditioner's vectors: stencil r, p_old read, p, q written;
    # update x, r, p, q read, x, r written; plus the M_e plane once per pass
    assert pb["survey"]["stencil"] == pytest.approx(4 * 8 + 4.0 / s)
    assert pb["survey"]["update"] == pytest.approx(6 * 8 + 4.0 / s)
    # stencil: edges w, a_old, a, q; nodes psi, b_old, b, G^T M p; packed masses (16 B per node)
    assert pb["kernel"]["stencil"] == pytest.approx(4 * 8 + 4 * node + 16.0 / 3.0 / s)
    # update, even iterations: edges w (r/w), q; diag K and M_e (4 B each); nodes v (r/w), G^T M p,
    # psi; W_n (4 B per node)
    even = 3 * 8 + 8.0 / s + 4 * node + 4.0 / 3.0 / s
    # odd iterations add the correction: edges x (r/w), a, a_prev; nodes x_n (r/w), b, b_prev
    odd = even + 4 * 8 + 4 * node
    assert pb["kernel"]["update"] == pytest.approx((even + odd) / 2)
    assert (even, odd) == (pytest.approx(35.6, abs=0.05), pytest.approx(78.3, abs=0.05))
