"""Shared pieces of the GPU parity tests: the oracle's response for given shifts and channel
weights, solved in parallel processes, and the per-channel bound with its achieved margins.

Parity is defined for fixed (xi, c): d[r, k] = sum_i Re(c[i, k] q_r^T (K - xi_i M)^{-1} f).
The bound per channel is |d_gpu - d_oracle| <= rel |d_oracle| + floor S_k with
S_k = sum_i |c[i, k] y_i|, y_i = q_r^T x_i (the size of the terms before they cancel).
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
    """Assert the per-channel bound; print the achieved margin and the plain relative error."""
    bound = rel * np.abs(d_ref) + floor * S
    err = np.abs(d_gpu - d_ref)
    ratio = err / bound
    plain = err / np.abs(d_ref)
    print(f"parity {label}: worst err/bound {ratio.max():.3g}, max plain rel err {plain.max():.3g} "
          f"(median {np.median(plain):.3g}), channels with plain rel err <= {rel:g}: "
          f"{int((plain <= rel).sum())}/{plain.size}")
    assert ratio.max() <= 1.0, f"{label}: worst err/bound {ratio.max():.3g}; max rel err {plain.max():.3g}"
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
