"""Shared pieces of the GPU parity tests: the oracle's response for given shifts and channel
weights, solved in parallel processes, and the per-channel bound with its achieved margins.

Parity is defined for fixed (xi, c): d[r, k] = sum_i Re(c[i, k] q_r^T (K - xi_i M)^{-1} f).
Every channel must meet |d_gpu - d_oracle| <= rel |d_oracle| (rel = 1e-6 for FP64 paths, 1e-5
for mixed precision).  The printout adds the ratio to rel |d| + floor S_k, S_k =
sum_i |c[i, k] y_i| with y_i = q_r^T x_i, which shows how far each channel is from the level
where the cancellation among the pole terms would start to limit any FP64 computation.
"""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def _pool(n):
    """A spawn pool of n single-threaded processes (the processes are the parallelism; BLAS
    threads inside each would oversubscribe the cores many times over)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return ProcessPoolExecutor(max_workers=max(1, n), mp_context=mp.get_context("spawn"))


def _solve_y(args):
    hx, hy, hz, sigma, loop, z_loop, rx, origin, current, shift = args
    from oracle.solvers import solve_lu
    from oracle.tem import TEMProblem
    P = TEMProblem(hx, hy, hz, sigma, loop, z_loop, rx, current=current, origin=origin)
    return P.Q @ solve_lu(P.K, P.Md, P.f, shift)


def oracle_responses(cases, processes=None):
    """cases: (model, shifts, c, rx or None) tuples.  One sparse LU solve per (case, shift),
    spread over spawned processes.  Returns [(d, S)] in the order of the cases."""
    tasks, owner = [], []
    for q, (m, shifts, c, rx) in enumerate(cases):
        rx = m.rx if rx is None else rx
        for s in shifts:
            tasks.append((m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, rx, m.origin,
                          getattr(m, "current", 1.0), complex(s)))
            owner.append(q)
    n = processes or min(len(tasks), len(os.sched_getaffinity(0)))
    with _pool(n) as ex:
        ys = list(ex.map(_solve_y, tasks))
    out = []
    for q, (m, shifts, c, rx) in enumerate(cases):
        y = np.stack([ys[t] for t in range(len(tasks)) if owner[t] == q])     # (s, n_rx)
        d = np.einsum("ik,ir->rk", np.asarray(c), y).real
        S = np.einsum("ik,ir->rk", np.abs(c), np.abs(y))
        out.append((d, S))
    return out


def check(d_gpu, d_ref, S, rel, floor, label=""):
    """Assert the plain relative error |d_gpu - d_oracle| / |d_oracle| <= rel on every channel;
    print it beside the cancellation-aware ratio err / (rel |d| + floor S_k) as a diagnostic."""
    bound = rel * np.abs(d_ref) + floor * S
    err = np.abs(d_gpu - d_ref)
    ratio = err / bound
    plain = err / np.abs(d_ref)
    print(f"parity {label}: max plain rel err {plain.max():.3g} (median {np.median(plain):.3g}), "
          f"channels with plain rel err <= {rel:g}: {int((plain <= rel).sum())}/{plain.size}; "
          f"worst err / (rel |d| + floor S) {ratio.max():.3g}")
    assert plain.max() <= rel, f"{label}: max plain rel err {plain.max():.3g} > {rel:g}"
    return plain


def _adjoint_task(args):
    hx, hy, hz, sigma, loop, z_loop, rx, origin, shift, c_row, g = args
    from oracle.tem import TEMProblem
    P = TEMProblem(hx, hy, hz, sigma, loop, z_loop, rx, origin=origin)
    return P.adjoint_gradient([shift], c_row[None, :], g)


def oracle_adjoint(m, shifts, c, g, processes=None):
    """The oracle's J^T g = dphi/dlog sigma for dphi/dd = g (fixed): a sum over the shifts, so each
    shift is one process's task (its forward and adjoint solves by sparse LU)."""
    c = np.asarray(c)
    base = (m.hx, m.hy, m.hz, m.sigma, m.loop_xy, m.z_loop, m.rx, m.origin)
    n = processes or min(len(shifts), len(os.sched_getaffinity(0)))
    with _pool(n) as ex:
        return sum(ex.map(_adjoint_task, [base + (complex(s), c[i], g) for i, s in enumerate(shifts)]))
