#!/usr/bin/env python
"""Benchmark of the GB300 PAGANI engine: time-to-epsrel and integrand evals/s.

One step = one complete adaptive integration (every iteration of Algorithm 2,
all steps of the hot path) of each integral of the workload, through the C ABI
(pagani_integrate_ex).  Default workload: the 5-D Gaussian at epsrel 1e-7 and
the 6-D oscillatory integrand at epsrel 1e-8 (rel-err filtering off), plus the
same oscillatory integral at 1e-10, whose active set reaches the 1e6..1e7
regions the oscillatory workload is specified for (at 1e-8 it converges with
6.6e4); seeded synthetic parameters.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank integrates the same workload independently
(replicas: the method has no cross-GPU step on one box); value = all ranks'
evaluations / the slowest rank's time.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_DEFAULT = "gaussian_d5+oscillatory_d6+oscillatory_d6_1e-10"
METRIC = "integrand evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form and filtering-ablation reports")
    ap.add_argument("--no-scale", action="store_true", help="skip the 8-D C0 management-at-scale report")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation report")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle time budget per integral")
    ap.add_argument("--quiet", action="store_true")
    ap.add_argument("--paper-suite", action="store_true",
                    help="instead of the bench line: digits of precision reached on the paper's f1..f8 (Sec. 4.2)")
    return ap.parse_args()


def workloads(spec: str):
    from paper_2104_06494_gb300.workloads import config_workloads
    allw = config_workloads()
    return [allw[name] for name in spec.split("+")]


def npoints(n: int) -> int:
    return 1 + 8 * n + 6 * n * (n - 1) + 4 * n * (n - 1) * (n - 2) // 3 + 2 ** n


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                         if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------- oracle (CPU)
def oracle_sample(w, budget_s: float, gpu_trace=None):
    """The oracle on a bounded sample of one integral: its first k iterations
    (status it_max), k chosen so the work fits about budget_s seconds."""
    import numpy as np
    from oracle import capi
    t = time.perf_counter()
    r1 = capi.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions, relerr_filter=w.relerr_filter,
                        it_max=1)
    dt1 = time.perf_counter() - t
    rate = r1.n_regions / max(dt1, 1e-9)            # regions/s of the oracle on this integral
    k = 1
    if gpu_trace is not None and len(gpu_trace) > 1:
        cum = np.cumsum(gpu_trace["s"])
        k = int(max(1, np.searchsorted(cum, rate * budget_s, side="right")))
        k = min(k, len(gpu_trace))
    if k > 1:
        t = time.perf_counter()
        r = capi.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions,
                           relerr_filter=w.relerr_filter, it_max=k)
        dt = time.perf_counter() - t
    else:
        r, dt = r1, dt1
    return {"name": w.name, "iterations": r.iterations, "regions": r.n_regions,
            "evals": r.n_regions * npoints(w.dim), "seconds": dt, "status": r.status}


def cpu_baseline(ws, budget_s, gpu_traces):
    """(single-threaded baseline, OpenMP baseline): the oracle on a bounded
    sample of each integral, then the OpenMP build of the oracle (its
    per-region Evaluate loop on all host cores, every other step serial) on
    exactly the same sample."""
    from oracle import capi
    parts = [oracle_sample(w, budget_s, gpu_traces.get(w.name)) for w in ws]
    evals = sum(p["evals"] for p in parts)
    secs = sum(p["seconds"] for p in parts)
    sample = "; ".join(f"{p['name']}: first {p['iterations']} iterations ({p['regions']} regions, "
                       f"{p['seconds']:.1f} s)" for p in parts)
    single = {"value": evals / secs, "unit": METRIC, "cores": 1, "kind": "oracle",
              "sample": "single-threaded C oracle, " + sample}
    threads = int(capi._load(parallel=True).omp_get_max_threads())
    psecs = 0.0
    for w, p in zip(ws, parts):
        t = time.perf_counter()
        r = capi.integrate(w.family, w.dim, w.params, w.epsrel, w.epsabs, w.max_regions,
                           relerr_filter=w.relerr_filter, it_max=p["iterations"], parallel=True)
        psecs += time.perf_counter() - t
        assert r.n_regions == p["regions"], (w.name, r.n_regions, p["regions"])
    parallel = {"value": evals / psecs, "unit": METRIC, "cores": threads, "kind": "oracle (OpenMP Evaluate)",
                "sample": f"the same sample, OpenMP build of the C oracle on {threads} threads"}
    return single, parallel


# --------------------------------------------------------------- helpers
def source_hash() -> str:
    h = hashlib.sha256()
    for f in ("pagani_eval.cuh", "pagani_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2104_06494_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# DRAM bytes per evaluated region of k_evaluate_loop (read + write), from the
# ncu capture of the 5-D Gaussian's 262,144-region launch
# (profiles/k_evaluate_loop_gaussian_d5.md), keyed by the hash of the kernel
# sources it was taken on: the figure no longer applies once they change.
EVAL_DRAM_BYTES_PER_REGION = {
    # 13,118,464 B read + 22,528 B written over 262,144 regions (9th Evaluate
    # launch of the 5-D Gaussian at epsrel 1e-7)
    "8f3f041fb8363b6d": 50.13,
}


def traffic_bytes_per_region():
    """DRAM bytes per evaluated region of Evaluate for the current kernel
    sources, or None when they changed since the counters were taken."""
    return EVAL_DRAM_BYTES_PER_REGION.get(source_hash())


def differentiation_report(pg, torch, flush, reps: int = 3):
    """The differentiated form on the d = 6 parametric Gaussian next to the
    plain single integral at the same accuracy: forward with the leaf set kept,
    backward over it, and the gradient's error against the closed form."""
    import numpy as np
    from oracle import closed_forms as cf
    from paper_2104_06494_gb300.workloads import config_workloads
    w = config_workloads()["gaussian_d6_grad"]
    n, p = w.dim, np.array(w.params)

    def timed(fn):
        best = None
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b)
            best = t if best is None else min(best, t)
        return best, out
    stream = torch.cuda.current_stream().cuda_stream
    plain_ms, r0 = timed(lambda: pg.pagani_integrate_ex(n, w.family, p, w.epsrel, w.epsabs, w.max_regions,
                                                        stream=stream))
    fwd_ms, r = timed(lambda: pg.pagani_integrate_ex(n, w.family, p, w.epsrel, w.epsabs, w.max_regions,
                                                     stream=stream, keep_leaves=1))
    lower, level = pg.pagani_leaves(n)
    bwd_ms, (v, g) = timed(lambda: pg.pagani_gradient(n, w.family, p, lower, level, stream=stream))
    tot, gc = cf.gaussian_gradient(n, p)
    scale = np.concatenate([np.full(n, abs(tot)), p[:n] * abs(tot)])
    err = np.abs(g - np.array(gc))
    return {"workload": w.name, "theta": "a_1..a_6, w_1..w_6", "epsrel": w.epsrel,
            "grad_err_over_errorest_bound": float(np.max(err / grad_error_bound(r.errorest, p, n))),
            "plain_ms": plain_ms, "forward_keep_leaves_ms": fwd_ms, "backward_ms": bwd_ms,
            "n_leaves": r.n_leaves, "regions": r.n_regions, "status": r.status,
            "value_true_relerr": abs(r.estimate - tot) / abs(tot),
            "grad_max_err_vs_closed_form": float(np.max(np.abs(g - np.array(gc)) / scale)),
            "grad_err_scale": "|I| for d/da, a_j |I| for d/dw",
            "backward_evals_per_s": r.n_leaves * npoints(n) / (bwd_ms * 1e-3)}


def grad_error_bound(errorest, p, n):
    """The gradient's error bound implied by the integral's error estimate:
    the rule's error on a box of a Gaussian factor of width 1/a behaves like
    (a h)^10, so d/da_j of it is at most 10 errorest / a_j, and d/dw_j (a shift
    by a fraction of the width 1/a_j) at most 10 a_j errorest."""
    import numpy as np
    a = np.asarray(p[:n], dtype=float)
    return np.concatenate([10 * errorest / a, 10 * errorest * a])


def hbm_peak_gbs():
    """The measured HBM copy bandwidth from MEASURED_PEAKS.json when that
    file is present, else a fallback figure of 6.8 TB/s."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def management_bandwidth(part, hbm_peak):
    """Achieved HBM bandwidth of the region-management kernels over one
    host-driven integration: algorithmic bytes from the per-iteration trace
    (s regions, r rel-err actives, n_surv survivors, n axes, whether a
    threshold search succeeded) over the phase's CUDA-event time.
      probe: per pass, every region's classification byte and error, 9 s
             (the passes of each iteration are in the trace)
      count: the classification bytes, s; after a search also E of each
             rel-err active region and the byte of each region the
             threshold finished, 8 r + (r - n_surv)
      split: the classification byte read; per survivor K and V read, its
             bounds and levels (9n) read, V_p and both halves (2 * 9n)
             written; per finished region V, E and its n levels read (the
             finished sums): s + n_surv (17 + 27 n) + (s - n_surv)(16 + n)"""
    import numpy as np
    tr, n = part["trace"], part["dim"]
    s = tr["s"].astype(float)
    surv = tr["n_survivors"].astype(float)
    rel = tr["n_relerr_active"].astype(float)
    ok = tr["search_ok"].astype(bool)
    passes = tr["probe_passes"].astype(float)
    probe_b = float(np.sum(passes * 9 * s))
    fin = s - surv
    count_b = float(np.sum(s + np.where(ok, 8 * rel + (rel - surv), 0.0)))
    # the last iteration is split only when the loop goes on (not here: it ended)
    split_b = float(np.sum((s + surv * (17 + 27 * n) + fin * (16 + n))[:-1]))
    out = {}
    for key, b, ms in (("threshold_probe", probe_b, part["phase_ms"][1]), ("sums_count", count_b, part["phase_ms"][2]),
                       ("filter_split", split_b, part["phase_ms"][3])):
        gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else None
        out[f"{key}_gbs"] = gbs
        out[f"{key}_hbm_frac"] = gbs / hbm_peak if gbs is not None and hbm_peak else None
    out["probe_passes"] = int(np.sum(passes))
    out["hbm_peak_gbs"] = hbm_peak
    return out


def scale_report(pg, torch, flush, roofline, peaks, hbm_peak, name: str = "c0_d8"):
    """The region-management kernels at scale: the 8-D C0 workload (epsrel
    1e-6, a 4e8-region pool, 2e8 regions and more per iteration), one
    host-driven pass with CUDA events per phase, and its time to result
    through the graph loop."""
    from oracle import closed_forms as cf
    from paper_2104_06494_gb300.workloads import config_workloads
    w = config_workloads()[name]
    stream = torch.cuda.current_stream().cuda_stream
    pg.pagani_workspace_reserve(w.max_regions, w.dim)
    try:
        r = pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions,
                                   use_graph=0, trace=True, stream=stream)
        work = roofline.evaluate_work(w.family, w.dim, r.trace["s"])
        part = {"trace": r.trace, "dim": w.dim, "phase_ms": list(r.phase_ms)}
        pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions, stream=stream)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g = pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions, stream=stream)
        b.record()
        torch.cuda.synchronize()
        ttr = a.elapsed_time(b)
    finally:
        pg.pagani_workspace_release()
    ex = cf.closed_form(w.family, w.dim, w.params)
    achieved = work["flops"] / (r.eval_ms * 1e-3) / 1e12
    return {"workload": name, "epsrel": w.epsrel, "max_regions": w.max_regions, "status": g.status,
            "iterations": g.iterations, "regions": g.n_regions, "max_active": int(r.trace["s"].max()),
            "time_to_result_ms": ttr, "evals_per_s": g.n_regions * npoints(w.dim) / (ttr * 1e-3),
            "true_relerr": abs(g.estimate - ex) / abs(ex), "errorest_rel": g.errorest / abs(g.estimate),
            "within_errorest": bool(abs(g.estimate - ex) <= g.errorest),
            "evaluate_ms": r.eval_ms, "evaluate_fp64_frac": achieved / peaks["fma_tflops"],
            "cache_fill_ms": r.phase_ms[0], "threshold_probe_ms": r.phase_ms[1],
            "sums_count_ms": r.phase_ms[2], "filter_split_ms": r.phase_ms[3],
            "evaluate_share": r.eval_ms / (r.eval_ms + sum(r.phase_ms)),
            **management_bandwidth(part, hbm_peak)}


def filtering_report(pg, torch, flush, max_regions: int = 1 << 27):
    """The filtering ablation of Sec. 4.2 on the paper's own case, f4 in 8-D
    at three digits: Threshold-Classify with both triggers (the default), the
    memory trigger only, the unchanged-digits trigger only, and off."""
    from oracle import closed_forms as cf
    from paper_2104_06494_gb300.workloads import paper_integrands
    w = paper_integrands()["f4_d8"]
    ex = cf.closed_form(w.family, w.dim, w.params)
    stream = torch.cuda.current_stream().cuda_stream
    out = {"workload": "f4_d8 (Gaussian, a_j = 25, w_j = 1/2)", "epsrel": 1e-3, "max_regions": max_regions}
    for mode, name in ((1, "both_triggers"), (2, "memory_trigger_only"), (3, "digits_trigger_only"), (0, "off")):
        pg.pagani_integrate_ex(w.dim, w.family, w.params, 1e-3, max_regions=max_regions, heuristic_filter=mode,
                               stream=stream)            # warm-up: graph, workspace
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = pg.pagani_integrate_ex(w.dim, w.family, w.params, 1e-3, max_regions=max_regions,
                                   heuristic_filter=mode, stream=stream)
        b.record()
        torch.cuda.synchronize()
        out[name] = {"ms": a.elapsed_time(b), "status": r.status, "iterations": r.iterations,
                     "regions": r.n_regions, "true_relerr": abs(r.estimate - ex) / abs(ex),
                     "errorest_rel": r.errorest / abs(r.estimate)}
    return out


def batching_report(pg, torch, flush, slot: int = 16384):
    """The batched form: 4096 independent integrals (dimension 3..8, five
    families, epsrel 1e-4..1e-8, each with a pool of `slot` regions) in one
    graph launch, next to the same 4096 integrals as looped single calls with
    the same pool size."""
    import numpy as np
    from oracle import closed_forms as cf
    from paper_2104_06494_gb300.workloads import batch_workloads
    items = batch_workloads()
    pg.pagani_integrate_batch(items, slot)          # warm-up: workspace, autotune, graph
    flush.zero_()
    torch.cuda.synchronize()
    res, dev_ms = pg.pagani_integrate_batch(items, slot)
    t0 = time.perf_counter()
    res, _ = pg.pagani_integrate_batch(items, slot)
    batch_wall_ms = (time.perf_counter() - t0) * 1e3
    stream = torch.cuda.current_stream().cuda_stream
    for w in items[:32]:                             # warm the single-call graphs
        pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, slot, relerr_filter=w.relerr_filter,
                               stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    a.record()
    singles = [pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, slot,
                                      relerr_filter=w.relerr_filter, stream=stream) for w in items]
    b.record()
    torch.cuda.synchronize()
    loop_wall_ms = (time.perf_counter() - t0) * 1e3
    loop_dev_ms = a.elapsed_time(b)
    same = sum(int(r["status"] == g.status and r["n_regions"] == g.n_regions and
                   abs(r["estimate"] - g.estimate) <= 1e-12 * abs(g.estimate) + 1e-300)
               for r, g in zip(res, singles))
    ex = np.array([cf.closed_form(w.family, w.dim, w.params) for w in items])
    inside = np.abs(res["estimate"] - ex) <= res["errorest"]
    evals = int(sum(int(r["n_regions"]) * npoints(w.dim) for r, w in zip(res, items)))
    return {"items": len(items), "max_regions_per_item": slot, "batch_device_ms": dev_ms,
            "batch_wall_ms": batch_wall_ms, "looped_single_wall_ms": loop_wall_ms,
            "looped_single_device_ms": loop_dev_ms, "speedup_wall": loop_wall_ms / batch_wall_ms,
            "integrals_per_s": len(items) / (batch_wall_ms * 1e-3), "evals_per_s": evals / (dev_ms * 1e-3),
            "converged_integrals_per_s": int(np.sum(res["status"] == 0)) / (batch_wall_ms * 1e-3),
            "converged_outside_tau": int(np.sum((res["status"] == 0) &
                                                (np.abs(res["estimate"] - ex) >
                                                 np.maximum(res["errorest"],
                                                            np.array([w.epsrel for w in items]) * np.abs(ex))))),
            "items_equal_to_single_calls": same,
            "status_counts": {int(k): int(v) for k, v in zip(*np.unique(res["status"], return_counts=True))},
            "within_errorest_of_closed_form": float(inside.mean())}


def paper_suite_report(pg, torch, max_regions: int = 1 << 28, digits=range(3, 11)):
    """The accuracy experiment of Sec. 4.2 on the paper's fixed-parameter
    integrands f1..f8: each at epsrel 1e-3, 1e-4, ... until a run does not
    converge, with a pool of max_regions regions; time to result (CUDA
    events), status, iterations, regions, the error estimate and, where a
    closed form exists, the true relative error."""
    from oracle import closed_forms as cf
    from paper_2104_06494_gb300.workloads import paper_integrands
    stream = torch.cuda.current_stream().cuda_stream
    pg.pagani_workspace_reserve(max_regions, 8)
    out = {"max_regions": max_regions}
    for name, w in paper_integrands().items():
        ex = cf.closed_form(w.family, w.dim, w.params)
        runs = []
        for dg in digits:
            tau = 10.0 ** -dg
            kw = dict(max_regions=max_regions, relerr_filter=w.relerr_filter, stream=stream)
            pg.pagani_integrate_ex(w.dim, w.family, w.params, tau, **kw)  # warm-up: graph
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r = pg.pagani_integrate_ex(w.dim, w.family, w.params, tau, **kw)
            b.record()
            torch.cuda.synchronize()
            runs.append({"digits": dg, "ms": a.elapsed_time(b), "status": r.status, "iterations": r.iterations,
                         "regions": r.n_regions, "errorest_rel": r.errorest / abs(r.estimate),
                         "true_relerr": None if ex is None else abs(r.estimate - ex) / abs(ex),
                         "within_errorest": None if ex is None else bool(abs(r.estimate - ex) <= r.errorest)})
            if r.status != 0:
                break
        out[name] = runs
    pg.pagani_workspace_release()
    return out


def main():
    args = parse()
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    ws = workloads(args.workload)
    wl_name = args.workload

    if args.impl == "reference":
        # the reference arm of this build is the CPU oracle, on rank 0 only
        if rank != 0:
            if world > 1:
                dist.destroy_process_group()
            return
        from oracle import capi
        capi.build()
        step_secs, step_evals = [], []
        for i in range(args.warmup + args.steps):
            parts = [oracle_sample(w, args.cpu_seconds / 4) for w in ws]
            if i >= args.warmup:
                step_secs.append(sum(p["seconds"] for p in parts))
                step_evals.append(sum(p["evals"] for p in parts))
        value = sum(step_evals) / sum(step_secs)
        sample = "; ".join(f"{p['name']}: first {p['iterations']} iterations ({p['regions']} regions)" for p in parts)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(step_secs) / len(step_secs),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded splitmix64 parameters)",
                "config": {"workload": wl_name, "sample": "each step: the oracle's first iterations of every integral"},
                "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                                 "sample": "single-threaded C oracle, " + sample},
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        if world > 1:
            dist.destroy_process_group()
        return

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2104_06494_gb300 as pg
    from paper_2104_06494_gb300 import build as pbuild, roofline
    pbuild.build()
    pg.load()
    if args.paper_suite:
        if rank == 0:
            print(json.dumps({"paper_suite": paper_suite_report(pg, torch)}))
        if world > 1:
            dist.destroy_process_group()
        return
    stream = torch.cuda.current_stream(dev).cuda_stream

    # workspace outside the timed region (the paper times integration only)
    pg.pagani_workspace_reserve(max(w.max_regions for w in ws), max(w.dim for w in ws))
    peaks = pg.pagani_fp64_peak(stream)

    def run(w, **kw):
        return pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions,
                                      relerr_filter=w.relerr_filter, stream=stream, **kw)

    # one traced run per integral (untimed): iteration structure and results
    traced = {w.name: run(w, trace=True) for w in ws}
    # roofline of Evaluate: the same kernels, host-driven, CUDA events around
    # every Evaluate launch on the launching stream
    roof_parts = []
    hbm_peak, hbm_peak_source = hbm_peak_gbs()
    for w in ws:
        r = run(w, use_graph=0, trace=True)
        work = roofline.evaluate_work(w.family, w.dim, r.trace["s"])
        roof_parts.append({"name": w.name, "eval_ms": r.eval_ms, "launches": r.eval_launches,
                           "phase_ms": list(r.phase_ms), "dim": w.dim, "trace": r.trace, **work})
    fl = sum(p["flops"] for p in roof_parts)
    ins = sum(p["inst"] for p in roof_parts)
    ems = sum(p["eval_ms"] for p in roof_parts)
    nl = sum(p["launches"] for p in roof_parts)
    calls = {k: sum(p.get(k, 0) for p in roof_parts) for k in ("exp", "sincos", "div")}
    achieved = fl / (ems * 1e-3) / 1e12
    regions_per_launch = sum(int(traced[w.name].trace["s"].sum()) for w in ws) / nl
    per_region = traffic_bytes_per_region()
    traffic = per_region * regions_per_launch if per_region is not None else None
    # FP64 issue slots the algorithm needs, library calls at their measured cost
    fma_rate = peaks["fma_tflops"] * 1e12 / 2
    slots = ins + sum(calls[k] * fma_rate / (peaks[f"{k}_gps"] * 1e9) for k in calls)
    pipe_frac = slots / (ems * 1e-3) / fma_rate

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step():
        res = []
        for w in ws:
            res.append(run(w))
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    clocks = ClockSampler(gpu_index)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall0 = time.perf_counter()
    results = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        results.append(step())
        ev[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(step_ms) * 1e-3

    # e2e: the public call with host buffers, wall clock, copies included
    e2e_times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        for w in ws:
            pg.pagani_integrate_ex(w.dim, w.family, w.params, w.epsrel, w.epsabs, w.max_regions,
                                   relerr_filter=w.relerr_filter)
        e2e_times.append(time.perf_counter() - t0)

    evals_step = sum(r.n_regions * npoints(w.dim) for r, w in zip(results[0], ws))
    launches = sum(r.kernel_launches for res in results for r in res)
    h2d = sum(r.h2d_bytes for r in results[0])
    d2h = sum(r.d2h_bytes for r in results[0])
    t_max = dev_s
    e2e_s = sum(e2e_times)
    if world > 1:
        tt = torch.tensor([dev_s, e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max, e2e_s = float(tt[0]), float(tt[1])
    value = world * evals_step * args.steps / t_max
    e2e_value = world * evals_step * args.steps / e2e_s

    if rank == 0:
        from oracle import closed_forms as cf
        per = {}
        for w, r in zip(ws, results[0]):
            ex = cf.closed_form(w.family, w.dim, w.params)
            per[w.name] = {"dim": w.dim, "family": w.family, "epsrel": w.epsrel, "status": r.status,
                           "iterations": r.iterations, "regions": r.n_regions,
                           "estimate": r.estimate, "errorest": r.errorest,
                           "true_relerr": abs(r.estimate - ex) / abs(ex), "within_errorest": abs(r.estimate - ex) <= r.errorest,
                           "relerr_filter": w.relerr_filter}
        cpu = cpu_par = None
        if not args.no_cpu_baseline and world >= 1:
            cpu, cpu_par = cpu_baseline(ws, args.cpu_seconds, {w.name: traced[w.name].trace for w in ws})
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded splitmix64 parameters in the Genz-family ranges of the workloads)",
            "config": {"workload": wl_name, "time_to_result_ms": {n: None for n in per},
                       "integrals": per, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "wall_s": wall},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peaks["fma_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fma_tflops"], "traffic": traffic,
                         "regions_per_launch": regions_per_launch,
                         "traffic_source": "ncu DRAM bytes per region of this kernel source x regions per launch",
                         "kernel": "k_evaluate_loop", "peak_source": "measured FP64 FMA chain (pagani_fp64_peak)",
                         "avg_launch_ms": ems / nl, "flops_per_launch": fl / nl,
                         "fp64_issue_frac_est": pipe_frac, "library_calls_per_launch":
                             {k: v / nl for k, v in calls.items()},
                         "measured_rates_gps": {k: peaks[k] for k in ("exp_gps", "sincos_gps", "div_gps")},
                         "parts": [{k: p[k] for k in ("name", "eval_ms", "launches", "flops")} for p in roof_parts]},
            # per-phase device time of the same host-driven pass (the
            # performance breakdown of Sec. 4.2: evaluate / threshold search /
            # post-processing / filter and split)
            "breakdown": {p["name"]: {"evaluate_ms": p["eval_ms"], "cache_fill_ms": p["phase_ms"][0],
                                      "threshold_probe_ms": p["phase_ms"][1], "sums_count_ms": p["phase_ms"][2],
                                      "filter_split_ms": p["phase_ms"][3],
                                      "evaluate_share": p["eval_ms"] / (p["eval_ms"] + sum(p["phase_ms"])),
                                      **management_bandwidth(p, hbm_peak), "hbm_peak_source": hbm_peak_source}
                          for p in roof_parts},
            "clocks": clk,
            "gpu_launches": launches,
        }
        # time to result of each integral (device events, from a dedicated pass)
        for w in ws:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record()
            run(w)
            b.record()
            torch.cuda.synchronize()
            line["config"]["time_to_result_ms"][w.name] = a.elapsed_time(b)
        if not args.no_diff:
            line["differentiation"] = differentiation_report(pg, torch, flush)
        if not args.no_scale:
            pg.pagani_workspace_release()
            line["management_at_scale"] = scale_report(pg, torch, flush, roofline, peaks, hbm_peak)
        if not args.no_batch:
            line["batching"] = batching_report(pg, torch, flush)
            line["filtering"] = filtering_report(pg, torch, flush)
        if cpu is not None:
            line["cpu_baseline"] = cpu
            line["cpu_baseline_parallel"] = cpu_par
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
