"""Iteration counts and timings of the oracle's own iterative route (T2) on a whole model.

Test infrastructure (see ``oracle/__init__.py``): only ``tests/``, ``smoke()`` and the CPU legs of
``bench.py`` use this module.

T2 is the Jacobi-preconditioned COCG of ``solvers.solve_cocg`` (one shifted system of Eq. (rmj)
per pole, stopped on the FP64 residual recomputed from the iterate).  Like the paper's ``pmap``
over poles (Sec. 5.3), every shift runs in its own process, min(cores, s) processes at a time,
each with its own copy of the assembled system.  The poles are the oracle fitter's
(``rational.tem_poles_residues``), the model one of the seeded workloads.

``python -m oracle.t2_counts randblock128 [processes]`` writes
``oracle/t2_counts_<workload>.json``: per shift the iterations to ||f - A x|| <= 1e-12 ||f||,
the true relative residual reached and the seconds taken, plus the assembly time and the number
of processes.  The CPU baseline of ``bench.py`` scales its timed sample with these counts, so
the scale factor comes from the oracle itself.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _model(name):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2506_11657_gb300 import workloads as W   # seeded inputs only
    if name.startswith("randblock"):
        return W.randblock128(n=int(name[len("randblock"):]))
    return W.by_name(name)


def _solve_one(args):
    name, shift, tol = args
    from oracle.tem import TEMProblem
    from oracle.solvers import solve_cocg
    m = _model(name)
    t0 = time.perf_counter()
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    t1 = time.perf_counter()
    _, it, rel = solve_cocg(P.K, P.Md, P.f, shift, tol=tol, maxiter=40000)
    t2 = time.perf_counter()
    return {"shift": [shift.real, shift.imag], "iterations": int(it), "relres": float(rel),
            "assembly_s": t1 - t0, "solve_s": t2 - t1}


def count(name, processes=None, tol=1e-12):
    """Run T2 on every shift of workload `name`; returns the record that main() stores."""
    from oracle import rational as R
    m = _model(name)
    shifts, _, _ = R.tem_poles_residues(m.t, m.degree)
    cores = len(os.sched_getaffinity(0))
    nproc = min(processes or cores, len(shifts))
    # one thread per process: the processes are the parallelism (BLAS threads would oversubscribe)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(nproc) as pool:
        rows = pool.map(_solve_one, [(name, complex(s), tol) for s in shifts], chunksize=1)
    wall = time.perf_counter() - t0
    return {"workload": name, "tol": tol, "processes": nproc, "cores_available": cores, "wall_s": wall,
            "degree": m.degree, "shifts": rows,
            "iterations": [r["iterations"] for r in rows],
            "note": "T2 = oracle.solvers.solve_cocg (Jacobi-COCG, FP64), one process per shift"}


def _worker(conn, name, shifts):
    """One process of the sampler: assemble once, then time T2 solves capped at m iterations."""
    from oracle.tem import TEMProblem
    from oracle.solvers import solve_cocg
    m = _model(name)
    t0 = time.perf_counter()
    P = TEMProblem(m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, origin=m.origin)
    conn.send(time.perf_counter() - t0)
    while True:
        cmd = conn.recv()
        if cmd is None:
            break
        t0 = time.perf_counter()
        for sh in shifts:
            solve_cocg(P.K, P.Md, P.f, sh, tol=1e-300, maxiter=cmd)
        conn.send(time.perf_counter() - t0)
    conn.close()


class Sampler:
    """Bounded samples of T2 on every shift of one workload, the shifts spread over
    min(cores, s) persistent processes (each assembles its own system once).

    step(m) runs, in every process and for each of its shifts, one T2 solve capped at m
    iterations (so it includes the solver's set-up: the shifted matrix, r0, z0) and returns the
    wall time until the last process is done.  model_seconds() turns step(0) and step(m) timings
    into the time of a whole model: assembly + set-up + the largest per-process iteration total.
    """

    def __init__(self, name, shifts, processes=None):
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        self.cores_available = len(os.sched_getaffinity(0))
        n = min(processes or self.cores_available, len(shifts))
        self.groups = [list(range(q, len(shifts), n)) for q in range(n)]
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for g in self.groups:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_worker, args=(b, name, [complex(shifts[q]) for q in g]), daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)
        self.assembly_s = max(self._recv(c, 3600.0) for c in self.conns)

    def _recv(self, c, timeout):
        # a worker that died (or a wait past `timeout` seconds) raises instead of blocking forever
        t0 = time.perf_counter()
        while not c.poll(1.0):
            if any(not p.is_alive() for p in self.procs) or time.perf_counter() - t0 > timeout:
                self.close()
                raise RuntimeError("oracle sampler: a worker process died or stopped answering")
        return c.recv()

    @property
    def processes(self):
        return len(self.procs)

    def step(self, m):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(int(m))
        for c in self.conns:
            self._recv(c, 3600.0)
        return time.perf_counter() - t0

    def model_seconds(self, setup_s, step_s, m, iterations):
        """Whole-model time from a step(0) time, a step(m) time and per-shift iteration counts:
        the time of one shift-iteration (the most loaded process ran gmax shifts per step), and
        the shifts scheduled longest first over the processes, as a pool of one process per
        pole would run them."""
        gmax = max(len(g) for g in self.groups)
        per_iter = max(step_s - setup_s, 0.0) / (m * gmax)
        per_setup = setup_s / gmax
        load = [0.0] * self.processes
        for it in sorted(iterations, reverse=True):
            q = load.index(min(load))
            load[q] += per_setup + it * per_iter
        return self.assembly_s + max(load)

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()


def load_counts(name):
    """The stored record of count(name), or None."""
    path = os.path.join(HERE, f"t2_counts_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def main(argv):
    name = argv[1] if len(argv) > 1 else "randblock128"
    nproc = int(argv[2]) if len(argv) > 2 else None
    rec = count(name, nproc)
    out = os.path.join(HERE, f"t2_counts_{name}.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(out, rec["iterations"], f"{rec['wall_s']:.0f} s")


if __name__ == "__main__":
    main(sys.argv)
