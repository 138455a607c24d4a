#!/usr/bin/env python3
"""Benchmark: step-off TEM forward models per second on the 128^3 random-block model.

One step = one forward model through tem_forward (all shifted solves to an FP64 relative
residual of 1e-12, receiver projection and pole -> channel combination) with the grid,
conductivity and edge mass resident in HBM and the shared poles cached (they depend only on
the channel times and the degree).  The timed region holds exactly --steps forward models,
bracketed by a barrier and a device synchronisation, timed with CUDA events on the launching
stream; the working set (10 shifts x 6.4M edges, ~5.7 GB) is far larger than L2.

Extra keys: the FP64 path's models/s on the same model and its per-channel agreement with the
mixed path, per-step p50/p99, an end-to-end number through the C ABI from host buffers, the
roofline of the stencil pass (and of the update pass and the whole iteration), the derivative
actions on the 96^3 adjoint model, a continuous-batching sample of the serving stream, the CPU
oracle timed on a bounded sample with one process per shift, and the SM clocks sampled during
the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --serving-only --serve-requests 256     (the whole serving stream, one line)
Under torchrun each rank runs its own models (independent problems, no collective on the
data path); value = all ranks' models / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {"randblock128": 128, "randblock96": 96, "randblock64": 64}
METRIC = "TEM forward models/s at 128^3 (mixed precision, FP64 residual 1e-12)"
UNIT = "models/s"
HBM_FALLBACK_GBS = 6800.0
NODE = 8.0 / 3.0      # bytes per edge of one complex FP32 nodal vector (one entry per node)


def pass_bytes(s):
    """Bytes per interior edge per shift of one launch of each FP32 pass.

    "survey": the minimal two-pass COCG count -- the stencil reads r, p_old and writes p, q
    (32 B), the update reads x, r, p, q and writes x, r (48 B) -- plus the M_e plane, 4 B per
    edge per pass, amortised over the s shifts that sweep a tile together.
    "kernel": what the kernels move (ncu-verified): the same edge vectors plus the nodal
    vectors of the preconditioner, and the per-grid arrays (packed masses, diag K, M_e, W_n)
    read once per tile for all s shifts."""
    return {
        "survey": {"stencil": 32.0 + 4.0 / s, "update": 48.0 + 4.0 / s},
        "kernel": {
            # edges w, a_old read, a, q written; nodes psi, b_old read, b, G^T M p written; masses
            "stencil": 32.0 + 4 * NODE + (16.0 / 3.0) / s,
            # every iteration: edges w, q read, w written; diag K, M_e; nodes v, G^T M p read, v,
            # psi written; W_n.  Every other iteration also the correction of two iterations:
            # edges x, a, a_prev read, x written; nodes x_n, b, b_prev read, x_n written
            "update": 24.0 + 8.0 / s + 4 * NODE + (4.0 / 3.0) / s + (32.0 + 4 * NODE) / 2,
        },
    }


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            v = [x.strip() for x in ln.split(",")]
            if len(v) < 8:
                continue
            try:
                sm.append(float(v[0]))
                mx.append(float(v[1]))
            except ValueError:
                continue
            for n, val in zip(names, v[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


DATA = ("synthetic: seeded random-block conductivity (10 m cells, 8^3-cell blocks with "
        "log10 rho ~ U[0, 3], air on top), 200 m square loop, receiver at its centre")


def _config(workload, nside, model, n_shifts):
    """The workload both arms report: grid, poles, channels and the stopping rule."""
    return {"workload": workload, "grid": [nside] * 3, "cells_m": 10.0, "shifts": n_shifts,
            "degree": model.degree, "channels": len(model.t), "t_range_s": [float(f"{model.t[0]:.6g}"), float(f"{model.t[-1]:.6g}")],
            "tol": 1e-12, "l2": "working set ~5.7 GB at 128^3 >> L2 (no flush needed)"}


def _kernel_sha():
    h = hashlib.sha256()
    for f in ("kernels.cuh", "stencil_tma.cuh", "solver.cu"):
        with open(os.path.join(ROOT, "paper_2506_11657_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(which, units):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on today's kernels."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        if t.get("source_sha") != _kernel_sha():
            return None
        return float(t["kernels"][which]["dram_bytes_per_unit"] * units)
    except Exception:
        return None


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample(name, steps, warmup, m):
    """The oracle's iterative route (T2) on every shift of `name`, the shifts spread over
    min(cores, s) processes (the paper's one process per pole).  A step runs, in every process,
    T2 capped at m iterations for each of its shifts; step(0) gives the solver's set-up alone.
    The whole-model time is assembly + set-up + the oracle's own per-shift iteration counts
    (oracle/t2_counts_<name>.json, written by `python -m oracle.t2_counts <name>`) scheduled
    over the processes at the measured time per iteration.  Returns a dict, or None without
    the stored counts."""
    from oracle import rational as R
    from oracle import t2_counts as T
    from paper_2506_11657_gb300 import workloads as W
    rec = T.load_counts(name)
    if rec is None:
        return None
    model = W.randblock128(n=WORKLOADS[name])
    shifts, _, _ = R.tem_poles_residues(model.t, model.degree)
    S = T.Sampler(name, shifts)
    try:
        # the solver set-up alone, twice (its time is subtracted from every sample)
        setup = float(np.median([S.step(0) for _ in range(2)]))
        for _ in range(warmup):
            S.step(m)
        times = [S.step(m) for _ in range(steps)]
        model_s = S.model_seconds(setup, float(np.median(times)), m, rec["iterations"])
        return {"model_s": model_s, "step_s": times, "setup_s": setup, "assembly_s": S.assembly_s,
                "processes": S.processes, "cores_available": S.cores_available, "iterations": rec["iterations"],
                "m": m}
    finally:
        S.close()


def cpu_baseline_leg():
    """The CPU baseline of the GPU arm: the 128^3 sample (scaled to a whole model by the oracle's
    own iteration counts) and one whole 32^3 model of the same family solved end to end."""
    from oracle import t2_counts as T
    smp = oracle_sample("randblock128", steps=2, warmup=0, m=8)
    if smp is None:
        return None
    whole = T.count("randblock32")
    desc = (f"oracle T2 (Jacobi-COCG, FP64) on randblock128: {smp['processes']} processes, one per shift; "
            f"assembly {smp['assembly_s']:.1f} s, solver set-up {smp['setup_s']:.1f} s, then {smp['m']} "
            f"iterations of every shift ({smp['step_s'][0]:.2f} s); whole model = assembly + set-up + the "
            f"oracle's own T2 counts per shift (max {max(smp['iterations'])}, counted once by oracle.t2_counts) "
            f"at the measured time per iteration")
    return {"value": 1.0 / smp["model_s"], "unit": UNIT, "cores": smp["processes"],
            "cores_available": smp["cores_available"], "kind": "oracle", "sample": desc,
            "model_s_estimate": smp["model_s"],
            "whole_model_measured": {"workload": "randblock32 (32^3 cells, same recipe)", "processes": whole["processes"],
                                     "seconds": whole["wall_s"], "iterations": whole["iterations"]}}


def run_reference(args):
    """--impl reference: the CPU oracle, as it stands, on the same workload and metric.  Each
    step is a bounded sample (8 T2 iterations of every shift, one process per shift)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2506_11657_gb300 import workloads as W
    model = W.randblock128()
    t0 = time.perf_counter()
    smp = oracle_sample("randblock128", steps=args.steps, warmup=args.warmup, m=8)
    wall = time.perf_counter() - t0
    if smp is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle/t2_counts_randblock128.json is missing"}))
        return
    value = 1.0 / smp["model_s"]
    desc = (f"each step: 8 iterations of oracle T2 (Jacobi-COCG, FP64) on every shift of randblock128, "
            f"{smp['processes']} processes (one per shift); value = 1 / (assembly {smp['assembly_s']:.1f} s + "
            f"set-up {smp['setup_s']:.1f} s + the oracle's own T2 counts per shift at the measured time "
            f"per iteration)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(smp["step_s"])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": _config("randblock128", 128, model, len(smp["iterations"])),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": smp["processes"],
                             "cores_available": smp["cores_available"], "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving
def run_serving(n_req, stream):
    """Continuous batching on the first n_req requests of the seeded serving stream (grids of
    32^3..96^3, 16-20 poles): all arriving at once (capacity), then Poisson arrivals at 1.2x and
    0.5x that capacity (latency).  Beside it, the same requests one at a time through tem_forward
    in FP64 (the plain per-model GPU path)."""
    import torch
    from paper_2506_11657_gb300 import tem, workloads as W
    from paper_2506_11657_gb300.serving import PoleCache, run_stream
    models = [m for _, m in W.serving_stream(n_requests=n_req, seed=4)]
    poles = PoleCache()
    for m in models:
        poles.get(m.t, m.degree)
    torch.cuda.synchronize()
    srv = tem.Server(stream=stream)
    _, sat = run_stream(srv, [(0.0, m) for m in models], poles)
    srv.close()
    cap = sat["models_per_s"]
    out = {"workload": "serving_stream", "requests": len(models), "grids": sorted(set(len(m.hx) for m in models)),
           "capacity_models_per_s": cap, "failed": sat["failed"]}
    for load in (1.2, 0.5):
        rng = np.random.default_rng(4)
        arr = np.cumsum(rng.exponential(1.0 / (load * cap), size=len(models)))
        s2 = tem.Server(stream=stream)
        _, lat = run_stream(s2, [(float(a), m) for a, m in zip(arr, models)], poles)
        s2.close()
        out[f"load_{load}x"] = {"arrival_rate_per_s": load * cap, "models_per_s": lat["models_per_s"],
                                "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"],
                                "mean_queue_ms": lat["mean_queue_ms"], "failed": lat["failed"]}
    t0 = time.perf_counter()
    for m in models:
        g = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma, stream=stream)
        sh, c = poles.get(m.t, m.degree)
        tem.forward(g, m.loop_xy, m.z_loop, m.rx, sh, c, tem.default_options(precision="fp64"), stream=stream)
        g.close()
    torch.cuda.synchronize()
    out["fp64_one_at_a_time_models_per_s"] = len(models) / (time.perf_counter() - t0)
    out["served_over_fp64"] = cap / out["fp64_one_at_a_time_models_per_s"]
    return out


# ------------------------------------------------------------------ derivatives
def run_derivatives(stream, dev):
    """The derivative actions of Sec. 4 on the 96^3 adjoint model (64 receivers, 20 poles, 31
    channels): J dm (tem_jvp) and J^T g (tem_adjoint), one batched solve each after a forward that
    keeps its solutions, timed with CUDA events, and the transpose gap <g, J dm> - <J^T g, dm>."""
    import torch
    from paper_2506_11657_gb300 import tem, workloads as W
    m = W.adjoint96()
    sh, c, _ = tem.poles_residues(m.t, m.degree)
    g = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma, stream=stream)
    opt = tem.default_options(precision="mixed", tol=1e-12)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    rk = tem.forward(g, m.loop_xy, m.z_loop, m.rx, sh, c, opt, stream=stream, keep_state=True)
    e[1].record(stream)
    rng = np.random.default_rng(7)
    dm = rng.standard_normal(m.sigma.size) * (m.sigma.ravel() > 1e-6)
    gres = rng.standard_normal(rk.d.shape)
    jd = rk.state.jvp(dm, stream=stream)
    e[2].record(stream)
    gr = rk.state.adjoint(gres, stream=stream)
    e[3].record(stream)
    torch.cuda.synchronize()
    rk.state.close()
    g.close()
    lhs, rhs = float(np.sum(gres * jd)), float(np.dot(gr, dm))
    return {"workload": "adjoint96", "receivers": int(len(m.rx)), "forward_ms": e[0].elapsed_time(e[1]),
            "jvp_ms": e[1].elapsed_time(e[2]), "adjoint_ms": e[2].elapsed_time(e[3]),
            "transpose_rel_gap": abs(lhs - rhs) / (np.sum(np.abs(gres * jd)) + np.sum(np.abs(gr * dm)))}


def run_single_time(stream):
    """Sec. 3.1's single-time baseline against the shared-pole family on the 64^3 random-block model
    (31 channels): the single-time approximant of degree 14 (7 shifts, 217 solves: each channel its
    own) and the shared-pole families of degree 20 (10 solves; the workload's) and 38 (19 solves;
    the degree the paper finds on par with single-time degree 14, Sec. 5), all mixed precision to
    an FP64 residual of 1e-12, timed with CUDA events; and how far each shared-pole response is from
    the single-time one per channel (the approximation error of the shared family: its uniform
    error is absolute, so the late channels, ~1e7 below the early ones, show it most)."""
    import torch
    from paper_2506_11657_gb300 import tem, workloads as W
    m = W.randblock128(n=64)
    g = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma, stream=stream)
    opt = tem.default_options(precision="mixed", tol=1e-12)
    xi1, c1, err1 = tem.poles_residues([1.0], 14)
    tem.forward(g, m.loop_xy, m.z_loop, m.rx, xi1, np.repeat(c1, len(m.t), 1), opt, stream=stream)   # warm
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    d_single, solves = tem.forward_single_time(g, m.loop_xy, m.z_loop, m.rx, m.t, xi1, c1[:, 0], opt, stream=stream)
    e[1].record(stream)
    torch.cuda.synchronize()
    out = {"workload": "randblock64", "channels": len(m.t),
           "single_time": {"degree": 14, "solves": solves, "uniform_err": err1, "ms": e[0].elapsed_time(e[1])}}
    for degree in (m.degree, 38):
        sh, c, err = tem.poles_residues(m.t, degree)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_shared = tem.forward(g, m.loop_xy, m.z_loop, m.rx, sh, c, opt, stream=stream).d
        e1.record(stream)
        torch.cuda.synchronize()
        rel = np.abs(d_shared - d_single) / np.abs(d_single)
        out[f"shared_poles_{degree}"] = {"degree": degree, "solves": len(sh), "uniform_err": err,
                                         "ms": e0.elapsed_time(e1), "max_rel_diff_vs_single_time": float(rel.max()),
                                         "median_rel_diff_vs_single_time": float(np.median(rel))}
    g.close()
    return out


def run_sources(stream, n_src=4):
    """Several loop sources (block f, Sec. 4) on the 64^3 model: n_src loops of 120-280 m solved as
    one batch of n_src x 10 shifted systems (tem_forward_sources) against n_src separate forwards,
    mixed precision to 1e-12, CUDA events; the batch reads the per-grid arrays once per tile for
    all systems."""
    import torch
    from paper_2506_11657_gb300 import tem, workloads as W
    m = W.randblock128(n=64)
    g = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma, stream=stream)
    opt = tem.default_options(precision="mixed", tol=1e-12)
    sh, c, _ = tem.poles_residues(m.t, m.degree)
    xn = m.origin[0] + np.concatenate(([0.0], np.cumsum(m.hx)))
    loops = []
    for side in np.linspace(120.0, 280.0, n_src):
        a = xn[np.argmin(np.abs(xn + side / 2))]
        b = xn[np.argmin(np.abs(xn - side / 2))]
        loops.append(np.array([[a, a], [b, a], [b, b], [a, b]]))
    tem.forward(g, loops[0], 0.0, m.rx, sh, c, opt, stream=stream)      # warm
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    D = tem.forward_sources(g, loops, 0.0, m.rx, sh, c, opt, stream=stream)
    e[1].record(stream)
    sep = [tem.forward(g, lp, 0.0, m.rx, sh, c, opt, stream=stream).d for lp in loops]
    e[2].record(stream)
    torch.cuda.synchronize()
    g.close()
    same = all(np.array_equal(D[j], sep[j]) for j in range(n_src))
    return {"workload": "randblock64", "sources": n_src, "systems_per_batch": n_src * len(sh),
            "batched_ms": e[0].elapsed_time(e[1]), "separate_ms": e[1].elapsed_time(e[2]),
            "bitwise_equal_to_separate": bool(same)}


def pass_roofline(tem, grid, model, shifts, stream, nside):
    """Per-launch timing of the two FP32 passes with all shifts active (tem_profile_passes: CUDA
    events on the launching stream, 20 iterations) and the roofline figures of both."""
    prof = tem.profile_passes(grid, model.loop_xy, model.z_loop, shifts, tem.PREC_MIXED, n_iter=20, stream=stream)
    peak, peak_kind = _peaks()
    units = prof["units"]
    s = len(shifts)
    pb = pass_bytes(s)
    tma = os.environ.get("TEM_FP32_STENCIL", "") != "pipe" and nside % 2 == 0

    def gbs(nbytes, ms):
        return nbytes * units / (ms * 1e-3) / 1e9

    def leg(which, ms):
        a = gbs(pb["survey"][which], ms)
        k = gbs(pb["kernel"][which], ms)
        return {"launch_ms": ms, "achieved": a, "frac": a / peak, "bytes_per_unit": pb["survey"][which],
                "kernel_bytes": {"bytes_per_unit": pb["kernel"][which], "achieved": k, "frac": k / peak},
                "traffic": _traffic(which, units)}

    st = leg("stencil", prof["stencil_ms"])
    up = leg("update", prof["update_ms"])
    it_ms = prof["stencil_ms"] + prof["update_ms"]
    it_survey = (pb["survey"]["stencil"] + pb["survey"]["update"])
    it_kernel = (pb["kernel"]["stencil"] + pb["kernel"]["update"])
    roofline = {"bound": "hbm", "kernel": "k_cocg_stencil_tma" if tma else "k_cocg_stencil_pipe",
                "achieved": st["achieved"], "peak": peak, "unit": "GB/s", "frac": st["frac"],
                "traffic": st["traffic"], "peak_source": peak_kind,
                "bytes_per_unit": st["bytes_per_unit"], "units_per_launch": units,
                "algorithmic_bytes_per_launch": st["bytes_per_unit"] * units, "launch_ms": st["launch_ms"],
                "kernel_bytes": st["kernel_bytes"], "stencil_ctas_per_sm": prof["stencil_ctas_per_sm"],
                "update": dict(up, kernel="k_cocg_update_vec" if tma else "k_cocg_update<float>"),
                "iteration": {"ms": it_ms, "achieved": gbs(it_survey, it_ms), "frac": gbs(it_survey, it_ms) / peak,
                              "kernel_bytes": {"achieved": gbs(it_kernel, it_ms), "frac": gbs(it_kernel, it_ms) / peak}},
                "residual_ms": prof["residual_ms"],
                "byte_counts": "achieved/frac: survey bytes (two-pass COCG vectors + M_e/s); kernel_bytes: what the "
                               "kernels move incl. the nodal preconditioner (ncu-verified)"}
    return roofline


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--workload", default="randblock128", choices=sorted(WORKLOADS))
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serving-only", action="store_true")
    ap.add_argument("--no-derivatives", action="store_true")
    ap.add_argument("--no-single-time", action="store_true")
    ap.add_argument("--passes-only", action="store_true", help="time the two FP32 passes only (no forward)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2506_11657_gb300 import build as B
    from paper_2506_11657_gb300 import tem, workloads as W
    if not os.path.exists(tem.LIB_PATH):
        B.build()
    tem.lib()
    stream = torch.cuda.current_stream(dev)
    if args.serving_only:
        if rank == 0:
            print(json.dumps({"serving": run_serving(args.serve_requests, stream)}), flush=True)
        return

    nside = WORKLOADS[args.workload]
    model = W.randblock128(n=nside)
    shifts, c, uerr = tem.poles_residues(model.t, model.degree)
    grid = tem.Grid(model.hx, model.hy, model.hz, model.origin, model.sigma, stream=stream)
    opt_mixed = tem.default_options(precision="mixed", tol=1e-12)
    opt_fp64 = tem.default_options(precision="fp64", tol=1e-12)
    if args.passes_only:
        # the pass timings alone (a short command to run under a profiler)
        if rank == 0:
            print(json.dumps({"workload": args.workload, "roofline": pass_roofline(tem, grid, model, shifts, stream,
                                                                                 nside)}), flush=True)
        return

    def fwd(opt, keep=False):
        return tem.forward(grid, model.loop_xy, model.z_loop, model.rx, shifts, c, opt, stream=stream,
                           keep_state=keep)

    for _ in range(args.warmup):
        fwd(opt_mixed)
    res = fwd(opt_mixed, keep=True)
    iters_mixed, relres_mixed = res.state.stats()
    res.state.close()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    n0 = tem.launch_count()
    ev[0].record(stream)
    outs = []
    for k in range(args.steps):
        outs.append(fwd(opt_mixed).d)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    n1 = tem.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = np.array([ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)])
    total_ms = float(ev[0].elapsed_time(ev[args.steps]))
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * args.steps / (total_ms / 1000.0)

    # FP64 path on the same model, and the per-channel agreement of the two
    fp64 = None
    if args.fp64_steps > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r64 = None
        for _ in range(args.fp64_steps):
            r64 = fwd(opt_fp64, keep=True)
        e1.record(stream)
        torch.cuda.synchronize()
        it64, rr64 = r64.state.stats()
        r64.state.close()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        d64, dm = r64.d, outs[-1]
        rel = np.abs(dm - d64) / np.abs(d64)
        fp64 = {"models_per_s": 1000.0 / ms64, "ms_per_model": ms64, "iters_per_shift": it64.tolist(),
                "max_rel_err_mixed_vs_fp64": float(rel.max()),
                "median_rel_err_mixed_vs_fp64": float(np.median(rel)),
                "channels_rel_le_1e-5": int((rel <= 1e-5).sum()), "channels": int(rel.size)}

    # all K field snapshots of the 128^3 model (the columns of S R): s complex FP64 read, K FP64 written per edge
    snaps = None
    if not args.no_derivatives:
        rk = fwd(opt_mixed, keep=True)
        U = torch.empty((len(model.t), 3 * model.sigma.size), dtype=torch.float64, device=dev)
        rk.state.fields(out=U, stream=stream)
        e3, e4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e3.record(stream)
        rk.state.fields(out=U, stream=stream)
        e4.record(stream)
        torch.cuda.synchronize()
        rk.state.close()
        del U
        fms = e3.elapsed_time(e4)
        fbytes = 3 * model.sigma.size * (16 * len(shifts) + 8 * len(model.t))
        snaps = {"ms_all_channels": fms, "gbs": fbytes / (fms * 1e-3) / 1e9}
    derivs = run_derivatives(stream, dev) if not args.no_derivatives else None
    single = run_single_time(stream) if not args.no_single_time else None
    sources = run_sources(stream) if not args.no_single_time else None

    # per-launch timing of the passes with all shifts active (CUDA events on the launching stream)
    roofline = pass_roofline(tem, grid, model, shifts, stream, nside)

    # end to end through the C ABI from host buffers: grid upload + forward + result read-back
    e2e_steps = args.e2e_steps
    h2d = model.sigma.nbytes + 8 * (len(model.hx) + len(model.hy) + len(model.hz) + 3)
    h2d += model.loop_xy.nbytes + model.rx.nbytes + shifts.nbytes + c.nbytes
    d2h = 8 * len(model.rx) * len(model.t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g2 = tem.Grid(model.hx, model.hy, model.hz, model.origin, model.sigma, stream=stream)
        tem.forward(g2, model.loop_xy, model.z_loop, model.rx, shifts, c, opt_mixed, stream=stream)
        g2.close()
    torch.cuda.synchronize()
    e2e = {"value": e2e_steps / (time.perf_counter() - t0) if e2e_steps else None, "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    serving = run_serving(args.serve_requests, stream) if args.serve_requests > 0 else None
    grid.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and nside == 128:
        cpu = cpu_baseline_leg()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": DATA, "config": _config(args.workload, nside, model, len(shifts)),
                "fit_uniform_err": uerr,
                "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
                "iters_per_shift_mixed": iters_mixed.tolist(), "relres_mixed": relres_mixed.tolist(),
                "fp64": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(n1 - n0), "clocks": clocks, "serving": serving,
                "derivatives": derivs, "field_snapshots": snaps, "single_time_baseline": single,
                "multiple_sources": sources}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
