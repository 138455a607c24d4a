"""Host logic without a GPU: the autograd wrapper, the request-stream driver and its pole
cache (each against a stand-in for the library), and the seeded workloads the benchmark and
its stored iteration counts depend on."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W


def test_autograd_backward_is_the_adjoint(monkeypatch):
    """With a linear stand-in d = A log sigma, backward must return A^T g and close the state."""
    from paper_2506_11657_gb300 import autograd
    rng = np.random.default_rng(2)
    A = rng.standard_normal((2 * 5, 12))
    closed = []

    class State:
        def adjoint(self, g):
            return A.T @ np.asarray(g).ravel()

        def close(self):
            closed.append(True)

    class Grid:
        def set_sigma(self, s):
            self.ls = np.log(s)

    grid = Grid()

    def forward(g, loop_xy, z_loop, rx, shifts, c, options, keep_state=False):
        assert keep_state
        return types.SimpleNamespace(d=(A @ g.ls).reshape(2, 5), status=0, state=State())

    monkeypatch.setattr(autograd.tem, "forward", forward)
    ls = torch.tensor(rng.standard_normal(12), dtype=torch.float64, requires_grad=True)
    d = autograd.TEMForward.apply(ls, grid, None, 0.0, None, None, None, None)
    assert np.allclose(d.detach().numpy(), (A @ ls.detach().numpy()).reshape(2, 5))
    g = torch.tensor(rng.standard_normal((2, 5)), dtype=torch.float64)
    (d * g).sum().backward()
    assert np.allclose(ls.grad.numpy(), A.T @ g.numpy().ravel())
    assert closed == [True]


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
