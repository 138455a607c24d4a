"""GPU tests of the continuous-batching server (tem_server_*).

* a request's result is bitwise the same alone, in a mix, and through tem_forward;
* every served result matches the oracle's response for the same shifts and weights;
* a request that arrives while another runs is admitted before the first finishes and the
  two overlap on the device;
* an HBM budget that holds one request at a time makes the second wait;
* bad input is rejected at submit time.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _models():
    a = W.uniform_model(24, 10.0, 6, 0.02, 80.0, 1e-5, 1e-3, 11, 12)
    b = W.uniform_model(20, 10.0, 5, 0.005, 60.0, 1e-5, 1e-3, 11, 10, ny=18, nz=22)
    rng = np.random.default_rng(9)
    c = W.uniform_model(16, 12.0, 4, 0.05, 48.0, 1e-5, 1e-3, 11, 13)
    c.sigma = c.sigma * np.where(c.sigma > 1e-6, 10 ** rng.uniform(-1, 1, c.sigma.shape), 1.0)
    return [a, b, c]


def _run(server, models, poles):
    tickets = [server.submit(m, *poles[i]) for i, m in enumerate(models)]
    out = {}
    for _ in range(10000):
        server.step()
        for i, t in enumerate(tickets):
            if i in out:
                continue
            r = server.poll(t)
            if r is not None:
                out[i] = r
        if len(out) == len(tickets):
            break
    return [out[i] for i in range(len(tickets))]


@pytest.fixture(scope="module")
def setup():
    from paper_2506_11657_gb300 import tem
    models = _models()
    poles = [tem.poles_residues(m.t, m.degree)[:2] for m in models]
    return tem, models, poles


def test_alone_mixed_and_forward_agree_bitwise(setup):
    tem, models, poles = setup
    mixed = _run(tem.Server(iters_per_step=16), models, poles)
    for i, m in enumerate(models):
        alone = _run(tem.Server(iters_per_step=16), [m], [poles[i]])[0]
        assert alone[1]["status"] == tem.TEM_OK and mixed[i][1]["status"] == tem.TEM_OK
        assert np.array_equal(alone[0], mixed[i][0]), i
        grid = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
        ref = tem.forward(grid, m.loop_xy, m.z_loop, m.rx, poles[i][0], poles[i][1],
                          tem.default_options(precision="mixed")).d
        assert np.array_equal(ref, mixed[i][0]), i


def test_served_results_match_the_oracle(setup):
    """Each served result -- the three requests in one mix, and each alone -- against the
    oracle's sparse-LU response for the same shifts and weights, with the bound of the mixed
    forward tests (rel 1e-5, cancellation floor 1e-9 S_k)."""
    from tests._parity import check, oracle_responses
    tem, models, poles = setup
    refs = oracle_responses([(m, poles[i][0], poles[i][1], None) for i, m in enumerate(models)])
    mixed = _run(tem.Server(iters_per_step=16), models, poles)
    for i, m in enumerate(models):
        alone = _run(tem.Server(iters_per_step=16), [m], [poles[i]])[0]
        d_ref, S = refs[i]
        for label, res in (("mixed", mixed[i]), ("alone", alone)):
            assert res[1]["status"] == tem.TEM_OK
            check(res[0], d_ref, S, 1e-5, 1e-9, f"served {label} model {i}")


def test_late_request_is_admitted_while_another_runs(setup):
    tem, models, poles = setup
    big = W.uniform_model(40, 10.0, 10, 0.01, 120.0, 1e-5, 1e-2, 11, 16)
    pb = tem.poles_residues(big.t, big.degree)[:2]
    srv = tem.Server(iters_per_step=8)
    ta = srv.submit(big, *pb)
    srv.step()
    srv.step()
    assert srv.counts()[1] == 1
    tb = srv.submit(models[2], *poles[2])
    res = {}
    for _ in range(20000):
        srv.step()
        for k, t in (("a", ta), ("b", tb)):
            if k not in res:
                r = srv.poll(t)
                if r is not None:
                    res[k] = r
        if len(res) == 2:
            break
    sa, sb = res["a"][1], res["b"][1]
    assert sb["admit_s"] < sa["done_s"], "the late request waited for the running one"
    assert sb["done_s"] < sa["done_s"], "the small late request should finish first"


def test_budget_admits_one_at_a_time(setup):
    tem, models, poles = setup
    probe = tem.Server()
    t = probe.submit(models[0], *poles[0])
    probe.step()
    fp = None
    for _ in range(10000):
        r = probe.poll(t)
        if r is not None:
            fp = r[1]["footprint_bytes"]
            break
        probe.step()
    srv = tem.Server(hbm_budget_bytes=int(fp * 1.5), iters_per_step=16)
    out = _run(srv, [models[0], models[0]], [poles[0], poles[0]])
    s1, s2 = out[0][1], out[1][1]
    assert s2["admit_s"] >= s1["done_s"]
    assert np.array_equal(out[0][0], out[1][0])


def test_submit_rejects_bad_input(setup):
    tem, models, poles = setup
    m = _models()[0]
    m.sigma = m.sigma.copy()
    m.sigma.flat[3] = -1.0
    srv = tem.Server()
    with pytest.raises(tem.TEMError) as e:
        srv.submit(m, *poles[0])
    assert e.value.code == tem.TEM_EINVAL
