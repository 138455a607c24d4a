"""Drive the continuous-batching server with a stream of timed requests.

Requests arrive at given times (seconds from the start); each is submitted once the wall
clock passes its arrival time, and the server is stepped until every request has finished.
Latency = completion - arrival.  The shared poles depend only on the channel times and the
degree, so they are computed once per (times, degree) and reused.
"""
from __future__ import annotations

import time

import numpy as np

from . import tem


class PoleCache:
    def __init__(self):
        self._c = {}

    def get(self, t, degree):
        key = (tuple(np.round(np.log10(t), 12)), int(degree))
        if key not in self._c:
            sh, c, err = tem.poles_residues(t, degree)
            self._c[key] = (sh, c)
        return self._c[key]


def run_stream(server: tem.Server, items, poles: PoleCache | None = None, clock=time.perf_counter,
               sleep=time.sleep, max_wall_s=3600.0):
    """items: list of (arrival_s, workloads.Model).  Returns (results, summary) where results[q]
    = dict(d, latency_s, queue_s, stats) in input order."""
    poles = poles or PoleCache()
    order = sorted(range(len(items)), key=lambda q: items[q][0])
    t0 = clock()
    nxt = 0
    tickets = {}
    results = [None] * len(items)
    pending = set()
    while nxt < len(order) or pending:
        now = clock() - t0
        if now > max_wall_s:
            raise RuntimeError("run_stream: wall-clock limit reached")
        while nxt < len(order) and items[order[nxt]][0] <= now:
            q = order[nxt]
            arr, model = items[q]
            sh, c = poles.get(model.t, model.degree)
            tk = server.submit(model, sh, c)
            tickets[tk] = (q, arr)
            pending.add(tk)
            nxt += 1
        if pending:
            server.step()
            for tk in list(pending):
                r = server.poll(tk)
                if r is None:
                    continue
                d, stats = r
                q, arr = tickets[tk]
                done = clock() - t0
                results[q] = {"d": d, "latency_s": done - arr, "arrival_s": arr, "done_s": done,
                              "queue_s": stats["admit_s"] - stats["submit_s"], "stats": stats}
                pending.discard(tk)
        elif nxt < len(order):
            sleep(max(0.0, min(0.05, items[order[nxt]][0] - (clock() - t0))))
    wall = clock() - t0
    lat = np.array([r["latency_s"] for r in results])
    summary = {"requests": len(items), "wall_s": wall, "models_per_s": len(items) / wall,
               "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "mean_queue_ms": float(np.mean([r["queue_s"] for r in results]) * 1e3),
               "failed": int(sum(r["stats"]["status"] not in (tem.TEM_OK,) for r in results))}
    return results, summary
