#!/usr/bin/env python3
"""Throughput of the improved Yau--Yau filter's online stage on GB300.

One step = prediction (multi-scale kernel sum) + correction + normalisation + estimate
+ restart test (and a restart when it fires), for one trajectory of the workload.
Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision bf16|f32|f64] [--impl yy|reference]

Under torchrun (N > 1) every rank runs an independent trajectory of the same workload
(different seed); the path shards by trajectory with no collective, so the value is the
sum of trajectory-steps per second over ranks (weak scaling).  --shard rows instead splits
one filter's target rows across the ranks (all-gathers of rows and records every step;
strong scaling).  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import WORKLOADS, simulate, sobol_poly_params, sobol_scramble_params  # noqa: E402
from synth.configs import batched_workloads  # noqa: E402

DEFAULT_WORKLOAD = "cubic_r1000_n65536"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the prediction
# kernel, from one ncu capture of the workload, keyed by workload, screen operands and
# whether the kernel ran on CTA pairs.  An entry is removed whenever the kernel changes
# after its capture.
NCU_TRAFFIC = {("cubic_r1000_n65536", "fp8", False): 39.310848e6 + 0.567552e6}
# --cta-pair: the tensor-core prediction on 2-CTA clusters (yy_set_cta_pair)
CTA_PAIR = False
METRIC = "filter steps/s & kernel pair-evals/s at r=1000: mixed vs FP32, same RMSE"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms.  Sampling is live before
    the region starts (the first sample has arrived); the summary keeps the samples read
    between mark_start() and one interval after mark_end() (all of them without marks)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_S = 0.1

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", str(int(self.INTERVAL_S * 1000))], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.monotonic() + 3.0
            while not self.lines and self.proc.poll() is None and time.monotonic() < deadline:
                time.sleep(0.01)
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()
        if self.proc is not None:   # let the sample covering the region's last interval arrive
            deadline = self.t1 + 2.5 * self.INTERVAL_S
            while time.monotonic() < deadline and not any(t > self.t1 for t, _ in self.lines):
                time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def _selected(self):
        if self.t0 is None or self.t1 is None:
            return [ln for _, ln in self.lines]
        inside = [ln for t, ln in self.lines if self.t0 <= t <= self.t1 + self.INTERVAL_S]
        if inside:
            return inside
        after = [ln for t, ln in self.lines if t >= self.t0]
        return after[:1]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self._selected():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    """(rank, world size, local rank, torch.distributed or None) from the torchrun
    environment; NCCL when CUDA is present, else gloo (host-side tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws, local, dist


def shard_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s trajectory: every rank filters its own independent trajectory
    (weak scaling; the path has no exchange step, so no collective in the data path)."""
    return base + 1000 * rank


def max_over_ranks(x: float, dist, device=None, dtype=None) -> float:
    """The largest value of x over all ranks (timed regions end when the slowest rank does)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([x], device=device if device is not None else "cpu", dtype=dtype or torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, t_max_s: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    return units_per_rank * ws / t_max_s


def _make_filter(w, precision, seed, device, stream=None, screen_prefix=0, screen_type="bf16"):
    from paper_2509_16896_gb300 import binding
    cfg = binding.config_from_workload(w, precision=precision, screen_prefix=screen_prefix, screen_type=screen_type)
    flt = binding.Filter(cfg, device=device, stream=stream)
    flt.init_nodes(sobol_poly_params(w.r, seed), sobol_scramble_params(w.r, seed), np.zeros(w.r))
    if precision == "bf16":
        flt.set_cta_pair(CTA_PAIR)
    return flt


def _gram_flops(r, k, stage, tiles, resc, bn=256):
    """Gram products the screen ran in one prediction: per screened block of 128 targets x
    bn sources 2 x 128 x bn x (stage k) flops for the first pass over the first stage k
    coordinates, plus 2 x 128 x bn x r for every block screened again over all of them."""
    r_pad = (r + 63) // 64 * 64
    return 2.0 * 128 * bn * (tiles * min(stage * k, r_pad) + resc * r_pad)


def _config(w, prec, screen_type):
    return {"workload": w.name, "r": w.r, "n": w.n, "n_scales": w.n_scales, "dt": w.dt,
            "R": w.R, "restart_interval": w.restart_interval, "ess_frac": w.ess_frac,
            "precision": prec, "trajectories_per_gpu": 1, "time_loop": "one CUDA graph of K steps",
            "screen_operands": screen_type if prec == "bf16" else None,
            "l2": f"inputs larger than L2 (u is {w.n * w.r * 4 / 1e6:.0f} MB)"
                  if w.n * w.r * 4 > 129e6 else
                  f"u ({w.n * w.r * 4 / 1e6:.1f} MB) fits in L2: steps follow each other, no flush"}


def _rmse(est, truth):
    K, r = truth.shape
    return float(np.sqrt(np.sum((est - truth) ** 2) / (K * r)))


def _tensor_peak(screen_type):
    peaks, src = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    note = f"{src}: bf16_tflops (burst; prediction launches timed alone)"
    if screen_type == "fp8":   # FP8 dense rate = 2 x BF16 (4.5 / 2.25 PFLOP/s nominal)
        peak, note = 2.0 * peak, f"{src}: 2 x bf16_tflops (fp8 nominal ratio; burst; prediction launches timed alone)"
    return peak, note


def _fma_peak():
    peaks, _ = _peaks()
    return 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def measure_single(w, prec, screen_type, screen_prefix, K, W, device, seed, dist=None, local=0):
    """One trajectory of workload w: K steps replayed as one CUDA graph after W untimed
    steps (CUDA events on the filter's stream, clocks sampled in the region), then the
    prediction launches timed alone for the dominant kernel's roofline.  Returns the
    result dict and the objects the end-to-end leg reuses."""
    import torch
    tr = simulate(w.model, w.r, W + K, w.dt, seed=seed)
    stream = torch.cuda.Stream(device)
    flt = _make_filter(w, prec, seed, device, stream, screen_prefix=screen_prefix, screen_type=screen_type)
    dys = torch.tensor(tr.dy, dtype=torch.float64, device=device)
    hist = torch.zeros((K, 2 * w.r + 4), dtype=torch.float64, device=device)
    with torch.cuda.stream(stream):
        if W:
            flt.run_steps(dys[:W])
        flt.graph_capture(dys[W:W + K], hist)   # captured, not executed, here
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = flt.launches()
    with ClockSampler(local) as clk:
        clk.mark_start()
        e0.record(stream)
        flt.graph_launch()
        e1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    if dist is not None:
        dist.barrier()
    launches = flt.launches() - l0
    ms = e0.elapsed_time(e1)
    t_max = max_over_ranks(ms, dist, device)
    h = hist.cpu().numpy()
    est = h[:, :w.r]
    rmse = _rmse(est, tr.x[W:W + K])
    restarts = int(h[:, 2 * w.r + 3].sum())
    # the dominant kernel: prediction launches from the state after the graph, timed alone
    n_pred = max(3, min(20, K))
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    pe0.record(stream)
    for _ in range(n_pred):
        flt.predict()
    pe1.record(stream)
    torch.cuda.synchronize()
    pred_ms = pe0.elapsed_time(pe1) / n_pred
    _, exact = flt.counters()
    _, mask = flt.get_nodes()
    live = int(w.n - mask.sum())
    screen = None
    stage = 128 if screen_type == "fp8" else 64
    if prec == "bf16":
        last, nxt, tiles, resc = flt.screen()
        screen = {"operands": screen_type, "first_pass_stages": last, "stage_coords": stage,
                  "stages": ((w.r + 63) // 64 * 64 + stage - 1) // stage, "tiles": tiles,
                  "rescreened": resc, "exact_pairs": exact,
                  "cta_pairs": flt.set_cta_pair(CTA_PAIR)}   # 2-CTA clusters of the schedule (0: single CTAs)
        flops = _gram_flops(w.r, last, stage, tiles, resc)
        peak, note = _tensor_peak(screen_type)
        roof = {"bound": "tensor", "achieved": round(flops / (pred_ms / 1e3) / 1e12, 3), "peak": peak,
                "unit": "TFLOP/s", "kernel": "k_ksum_tc (screen Gram products of the prediction)",
                "kernel_ms": round(pred_ms, 4), "algorithmic_flops_per_launch": flops, "peak_source": note}
    else:
        flops = 3.0 * w.n * w.n * w.r
        roof = {"bound": "alu", "achieved": round(flops / (pred_ms / 1e3) / 1e12, 3), "peak": _fma_peak(),
                "unit": "TFLOP/s", "kernel": "k_ksum_simt (difference form)", "kernel_ms": round(pred_ms, 4),
                "algorithmic_flops_per_launch": flops,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock"}
    roof["frac"] = round(roof["achieved"] / roof["peak"], 4)
    with torch.cuda.stream(stream):
        flt.update(dys[0])   # leave the handle in a consistent state
    steps_per_s = K / (t_max / 1e3)
    res = {"value": steps_per_s, "ms_per_step": t_max / K, "rmse": rmse, "restarts": restarts, "est": est,
           "clocks": clk.summary(), "gpu_launches": int(launches), "screen": screen, "roofline": roof,
           # per step: every (target, source, scale) term is covered by the prediction; the
           # screen proves most of them negligible and evaluates the rest (the self terms of
           # the live nodes and the exact pairs) in float32
           "pairs_covered_per_step": float(w.n_scales) * w.n * w.n,
           "pairs_evaluated_per_step": float(w.n_scales) * (live + exact) if prec == "bf16" else
                                       float(w.n_scales) * w.n * w.n}
    return res, flt, tr, stream


def _time_precision(w, prec, steps, warmup, tr, device, screen_prefix=0):
    """Steps/s and RMSE of another precision of the same path over the first `steps` timed
    steps of the same trajectory."""
    import torch
    stream = torch.cuda.Stream(device)
    flt = _make_filter(w, prec, w.seed, device, stream, screen_prefix=screen_prefix)
    dys = torch.tensor(tr.dy, dtype=torch.float64, device=device)
    hist = torch.zeros((steps, 2 * w.r + 4), dtype=torch.float64, device=device)
    with torch.cuda.stream(stream):
        if warmup:
            flt.run_steps(dys[:warmup])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        flt.run_steps(dys[warmup:warmup + steps], hist)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    est = hist.cpu().numpy()[:, :w.r]
    return {"precision": prec, "steps": steps, "ms_per_step": round(ms, 3),
            "value": round(1e3 / ms, 4), "unit": "filter steps/s",
            "rmse": _rmse(est, tr.x[warmup:warmup + steps])}


def _comparators(w, K, W, tr, device, fp32_steps, est):
    """The plain FP32 GPU form (every pair, difference form) and the screened FP32 form
    (the same kind of screen with its bound on the FMA pipes), each with its RMSE next to
    the mixed path's on the same steps: the first isolates pruning + precision, the second
    precision alone."""
    S = min(fp32_steps, K)
    out = {}
    for key, prec in (("fp32_dense", "f32"), ("fp32_screened", "f32s")):
        c = _time_precision(w, prec, S, W, tr, device)
        c["rmse_mixed_same_steps"] = _rmse(est[:S], tr.x[W:W + S])
        out[key] = c
    return out


def run_sharded(args):
    """One trajectory of the workload with its target rows split across the ranks (NCCL
    all-gathers of the rows and records every step); value = filter steps/s of that one
    filter (strong scaling)."""
    import torch
    from paper_2509_16896_gb300 import binding, sharded
    rank, ws, local, dist = _dist()
    device = f"cuda:{local}"
    torch.cuda.set_device(device)
    w = WORKLOADS[args.workload]
    prec = args.precision or w.precision
    W, K = args.warmup, args.steps
    tr = simulate(w.model, w.r, W + K, w.dt, seed=w.seed)
    cfg = binding.config_from_workload(w, precision=prec, screen_type=args.screen_type or w.screen_type)
    sf = sharded.ShardedFilter(cfg, dist, device)
    sf.init_nodes(sobol_poly_params(w.r, w.seed), sobol_scramble_params(w.r, w.seed), np.zeros(w.r))
    dys = torch.tensor(tr.dy, dtype=torch.float64, device=device)
    for k in range(W):
        sf.step(dys[k])
    est = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.mark_start()
        t0 = time.perf_counter()
        for k in range(W, W + K):
            sf.step(dys[k])
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        clk.mark_end()
    t_max = max_over_ranks(t, dist, device)
    mean, var, ess, z = sf.estimate()
    if rank == 0:
        out = {"metric": METRIC, "value": round(K / t_max, 4), "unit": "filter steps/s", "n_gpus": ws, "steps": K,
               "warmup": W, "ms_per_step": round(1e3 * t_max / K, 4), "higher_is_better": True, "scaling": "strong",
               "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded Euler-Maruyama cubic sensor, scrambled Sobol nodes)",
               "config": dict(_config(w, prec, args.screen_type or w.screen_type), partition="target rows split, "
                              "source set replicated; per step all-gather of rows and records"),
               "clocks": clk.summary(), "timing": "host wall clock around the K steps (NCCL in the loop)"}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_yy(args):
    import torch
    rank, ws, local, dist = _dist()
    device = f"cuda:{local}"
    torch.cuda.set_device(device)
    w = WORKLOADS[args.workload]
    prec = args.precision or w.precision
    if args.screen_type is None:
        args.screen_type = w.screen_type
    seed = shard_seed(w.seed, rank)
    W, K = args.warmup, args.steps
    res, flt, tr, stream = measure_single(w, prec, args.screen_type, args.screen_prefix, K, W, device, seed,
                                          dist, local)
    # ---- end to end through the C ABI with host buffers ---------------------------
    n_e2e = max(3, min(K, 50))
    dy_host = torch.tensor(tr.dy, dtype=torch.float64).pin_memory()
    dy_dev = torch.empty(w.r, dtype=torch.float64, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        with torch.cuda.stream(stream):
            dy_dev.copy_(dy_host[k % dy_host.shape[0]], non_blocking=True)
        flt.predict()
        flt.update(dy_dev)
        flt.estimate()
        flt.restart(mode=0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = whole_job_rate(n_e2e, ws, max_over_ranks(e2e_s, dist, device))
    steps_per_s = whole_job_rate(K, ws, K / res["value"])
    # ---- the other single-GPU workloads as sub-lines (rank 0 of a default run only) ----
    subs = {}
    if args.sublines and args.workload == DEFAULT_WORKLOAD and rank == 0:
        w2 = WORKLOADS["cubic_r100_n16384"]
        K2 = max(K, 20)
        r2, f2, tr2, _ = measure_single(w2, "bf16", w2.screen_type, 0, K2, W, device, w2.seed)
        est2 = r2.pop("est")
        sub = {"metric": "filter steps/s", "value": round(r2["value"], 3), "unit": "filter steps/s", "steps": K2,
               "config": _config(w2, "bf16", w2.screen_type), **{k: v for k, v in r2.items() if k != "value"}}
        if args.fp32_steps > 0:
            sub.update(_comparators(w2, K2, W, tr2, device, args.fp32_steps, est2))
        del f2
        sub["schedules"] = compare_schedules(w2, device, predicts_per_build=3)
        subs["cubic_r100_n16384"] = sub
        we = WORKLOADS["paper_e1_r1000_n2000"]
        re_, fe, tre, _ = measure_single(we, we.precision, we.screen_type, 0, we.steps, W, device, we.seed)
        re_.pop("est")
        del fe
        subs["paper_e1_r1000_n2000"] = {
            "metric": "filter steps/s", "value": round(re_["value"], 3), "unit": "filter steps/s", "steps": we.steps,
            "config": _config(we, we.precision, we.screen_type), **{k: v for k, v in re_.items() if k != "value"},
            "paper_context": {"note": "the paper's own time for this workload (1000 steps, r = 1000, n = 2000), "
                                      "MATLAB R2023b on an i9-12900K with one RTX 4090; context only",
                              "seconds_per_1000_steps": 150.54, "steps_per_s": 6.64, "rmse": 1.609}}
        subs["batched_256"] = measure_batch(max(W, 8), min(K, 20), device, "bf16", None, 0)
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    out = {
        "metric": METRIC,
        "value": round(steps_per_s, 4),
        "unit": "filter steps/s",
        "n_gpus": ws,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(1e3 / res["value"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        # screen operands + float32 exact evaluation, log-sum-exp and update
        "dtype": {"bf16": ("fp8+f32" if args.screen_type == "fp8" else "bf16+f32"), "f32": "f32",
                  "f32s": "f32", "f64": "f64"}[prec],
        "data": "synthetic (seeded Euler-Maruyama cubic sensor, scrambled Sobol nodes)",
        "config": _config(w, prec, args.screen_type),
        "pairs_covered_per_s": round(steps_per_s * res["pairs_covered_per_step"], 1),
        "pairs_evaluated_per_s": round(steps_per_s * res["pairs_evaluated_per_step"], 1),
        "rmse": res["rmse"],
        "restarts": res["restarts"],
        "clocks": res["clocks"],
        "e2e": {"value": round(e2e_val, 4), "unit": "filter steps/s",
                "h2d_bytes_per_step": 8 * w.r, "d2h_bytes_per_step": 8 * (2 * w.r + 2) + 56},
        "gpu_launches": res["gpu_launches"],
        "screen": res["screen"],
        "roofline": dict(res["roofline"], traffic=NCU_TRAFFIC.get((w.name, args.screen_type, CTA_PAIR))
                         if prec == "bf16" else None),
    }
    if args.fp32_steps > 0 and prec == "bf16":
        out.update(_comparators(w, K, W, tr, device, args.fp32_steps, res["est"]))
    if subs:
        out["sublines"] = subs
    if args.cpu_baseline and ws == 1:   # the oracle's baseline runs at N = 1 only
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def compare_schedules(w, device, predicts_per_build: int):
    """The materialised schedule (the paper's offline operator, online log-domain product)
    against the recomputed prediction on workload w's state after a few steps: the
    library's tuner times recompute, build and apply and reports its choice for
    `predicts_per_build` predictions per node set."""
    import torch
    from paper_2509_16896_gb300 import binding
    cfg = binding.config_from_workload(w, precision="bf16", materialise=1)
    f = binding.Filter(cfg, device=device)
    f.init_nodes(sobol_poly_params(w.r, w.seed), sobol_scramble_params(w.r, w.seed), np.zeros(w.r))
    tr = simulate(w.model, w.r, 3, w.dt, seed=w.seed)
    f.run_steps(torch.tensor(tr.dy, dtype=torch.float64, device=device))
    torch.cuda.synchronize()
    choice, (re, bu, ap) = f.tune_materialise(predicts_per_build, reps=3)
    op_gb = w.n_scales * ((w.n + 255) // 256 * 256) ** 2 * 4 / 1e9
    f.close()
    return {"predicts_per_build": predicts_per_build, "recompute_ms": round(re, 4), "build_ms": round(bu, 4),
            "apply_ms": round(ap, 4), "materialised_chosen": bool(choice), "operator_gb": round(op_gb, 2),
            "apply_gbs": round(op_gb / (ap / 1e3), 1)}


class OracleSample:
    """The FP64 oracle as it stands, set up once on the workload (nodes, prior state,
    prepared drift) and timed on this host's cores on a bounded sample: the prediction for a
    block of target rows (at least 4 per core, one row per OpenMP chunk) against all n
    sources plus the O(n r) correction, scaled to one full step."""

    def __init__(self, w):
        from oracle import filter as F, sobol
        self.F = F
        self.w = w
        self.cores = os.cpu_count() or 1
        self.p = F.Problem(model=w.model, r=w.r, n=w.n, dt=w.dt, R=np.full(w.r, w.R), n_scales=w.n_scales,
                           model_a=w.model_a)
        _, u = sobol.nodes(sobol_poly_params(w.r, w.seed), sobol_scramble_params(w.r, w.seed), w.n, w.R)
        self.st = F.init_state(self.p, u, np.zeros(w.r))
        self.prep = F.prepare(self.p, u, self.st.centre)
        self.dy = simulate(w.model, w.r, 1, w.dt, seed=w.seed).dy[0]
        t0 = time.perf_counter()
        F.predict(self.p, self.prep, self.st.logw, 0, self.cores, n_threads=self.cores)
        self.t_row = max(time.perf_counter() - t0, 1e-6) / self.cores

    def step_rate(self, seconds: float, threads: int | None = None):
        F, w = self.F, self.w
        th = threads or self.cores
        # t_row: seconds per row with every core busy; a single thread takes cores x longer
        per_row = self.t_row * (self.cores / th)
        rows = int(min(w.n, max(4 * th if th > 1 else 1, math.floor(seconds / per_row))))
        t0 = time.perf_counter()
        F.predict(self.p, self.prep, self.st.logw, 0, rows, n_threads=th)
        t_pred = time.perf_counter() - t0
        t0 = time.perf_counter()
        lw = F.log_likelihood(self.p, self.prep.x, self.dy) + self.st.logw
        lam, lh = F.normalise(lw)
        F.estimate(self.prep.x, lh)
        t_upd = time.perf_counter() - t0
        step_s = t_pred * (w.n / rows) + t_upd
        return {"value": round(1.0 / step_s, 6), "unit": "filter steps/s", "cores": th,
                "kind": "oracle",
                "sample": f"prediction of {rows} of {w.n} target rows (all sources, {w.n_scales} scales; "
                          f"one row per OpenMP chunk over {th} threads) + one full correction/estimate, "
                          f"scaled to one step; {t_pred + t_upd:.1f} s of CPU work"}


def cpu_baseline(w, seconds: float):
    orc = OracleSample(w)
    out = orc.step_rate(seconds)
    single = orc.step_rate(max(1.0, seconds / 4), threads=1)
    out["single_core_value"] = single["value"]
    out["single_core_sample"] = single["sample"]
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    prec = args.precision or w.precision
    t0 = time.perf_counter()
    orc = OracleSample(w)
    # each step: a sample of about 1 s of oracle work (the whole run stays within minutes)
    per_step = min(2.0, max(0.5, args.cpu_seconds / max(args.steps, 1)))
    for _ in range(args.warmup):
        orc.step_rate(0.2)
    vals = [orc.step_rate(per_step) for _ in range(args.steps)]
    v = statistics.median([x["value"] for x in vals])
    out = {"metric": METRIC, "impl": "reference", "value": v, "unit": "filter steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 / v, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Euler-Maruyama cubic sensor, scrambled Sobol nodes)",
           "config": _config(w, prec, args.screen_type or w.screen_type),
           "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "sample": vals[-1]["sample"], "value": v},
           "e2e": {"value": v, "unit": "filter steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": round(time.perf_counter() - t0, 2)}
    print(json.dumps(out), flush=True)


def measure_batch(S, K, device, prec, dist, local, rank=0):
    """256 ragged trajectories (r in 10..200, n log-uniform in 2048..32768, half cubic, half
    linear-Gaussian) advanced as one batch; value = trajectory-steps per second.  S untimed
    steps (at least 8, so that the autotuner routes on posteriors that have spread out),
    then the autotuner, then K steps as one CUDA graph."""
    import torch
    from paper_2509_16896_gb300 import binding
    members = batched_workloads(256, seed=shard_seed(4, rank), steps=S + K)
    cfgs = [binding.config_from_workload(m, precision=prec) for m in members]
    bt = binding.Batch(cfgs, device=device)
    trs = []
    for b, m in enumerate(members):
        bt.filters[b].init_nodes(sobol_poly_params(m.r, m.seed), sobol_scramble_params(m.r, m.seed), np.zeros(m.r))
        trs.append(simulate(m.model, m.r, S + K, m.dt, seed=m.seed, model_a=m.model_a))
    dy_all = torch.tensor(np.concatenate([t.dy for t in trs], axis=1), dtype=torch.float64, device=device)
    hist = torch.zeros((K, bt.H), dtype=torch.float64, device=device)
    with torch.cuda.stream(bt.stream):
        bt.run_steps(dy_all[:S])
    torch.cuda.synchronize()
    t_tune = time.perf_counter()
    bn, grid = bt.autotune(None, reps=2)
    t_tune = time.perf_counter() - t_tune
    routing = bt.routing()
    with torch.cuda.stream(bt.stream):
        bt.graph_capture(dy_all[S:S + K], hist)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = bt.launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.mark_start()
        e0.record(bt.stream)
        bt.graph_launch()
        e1.record(bt.stream)
        torch.cuda.synchronize()
        clk.mark_end()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, device)
    launches = bt.launches() - l0
    # the batched prediction alone
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(bt.stream)
    for _ in range(3):
        bt.predict()
    p1.record(bt.stream)
    torch.cuda.synchronize()
    pred_ms = p0.elapsed_time(p1) / 3
    # executed work of the last prediction: Gram products of the screened members (their
    # screen runs one full-coordinate pass), difference-form flops of the FP32-form members
    tflops, aflops = 0.0, 0.0
    for b, m in enumerate(members):
        if routing[b] == 0:
            last, _, tiles, resc = bt.filters[b].screen()
            tflops += _gram_flops(m.r, last, 64, tiles, resc, bn)
        else:
            aflops += 3.0 * m.n * m.n * m.r
    h = hist.cpu().numpy()
    rm_c, rm_l = [], []
    for b, (m, t) in enumerate(zip(members, trs)):
        est = h[:, bt.hist_off[b]:bt.hist_off[b] + m.r]
        rm = _rmse(est, t.x[S:S + K])
        (rm_c if m.model == "cubic" else rm_l).append(rm)
    peak, note = _tensor_peak("bf16")
    achieved = tflops / (pred_ms / 1e3) / 1e12
    bt.close()
    return {"metric": "trajectory-steps/s, 256 ragged filters in one batch",
            "value": round(256 * K / (ms / 1e3), 2), "unit": "trajectory-steps/s", "steps": K, "warmup": S,
            "ms_per_step": round(ms / K, 4), "dtype": prec,
            "config": {"workload": "batched_256", "trajectories": 256, "r": "10..200", "n": "2048..32768 log-uniform",
                       "n_scales": 2, "schedule": {"bn": bn, "grid": grid, "autotune_s": round(t_tune, 2),
                                                   "fp32_form_members": int(routing.sum()),
                                                   "fp32_form_max_r": int(max([m.r for m, p in zip(members, routing) if p] or [0]))},
                       "time_loop": "one CUDA graph of K batched steps"},
            "gpu_launches": int(launches), "clocks": clk.summary(),
            "rmse_cubic_mean": float(np.mean(rm_c)), "rmse_linear_mean": float(np.mean(rm_l)),
            "roofline": {"bound": "tensor", "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "kernel": "batched prediction (screen Gram products of the tensor-core members over the "
                                   "whole prediction, FP32-form members included in the time)",
                         "kernel_ms": round(pred_ms, 4), "algorithmic_flops_per_launch": tflops,
                         "fp32_form_flops_per_launch": aflops, "peak_source": note}}


def run_batch(args):
    import torch
    rank, ws_, local, dist = _dist()
    device = f"cuda:{local}"
    torch.cuda.set_device(device)
    res = measure_batch(max(args.warmup, 8), args.steps, device, args.precision or "bf16", dist, local, rank)
    if rank != 0:
        return
    res["value"] = round(res["value"] * ws_, 2)   # every rank advanced its own 256 members
    out = {"metric": res.pop("metric"), "value": res.pop("value"), "unit": res.pop("unit"), "n_gpus": ws_,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic (seeded Euler-Maruyama cubic sensor / linear-Gaussian, scrambled Sobol nodes)", **res}
    print(json.dumps(out), flush=True)


def run_learned(args):
    """Learned restart workload (r = 50, n = 8192, 500 steps, frequent ESS restarts): trains
    the proposal network on plain-run restarts of 64 training trajectories (seeds 100..163)
    and runs the held-out trajectory (seed 5) with both rules."""
    import torch
    from paper_2509_16896_gb300 import learned_restart as LR
    rank, ws_, local, dist = _dist()
    if rank != 0:
        return   # a quality comparison on one GPU: the other ranks do no work
    device = f"cuda:{local}"
    torch.cuda.set_device(device)
    w = WORKLOADS["cubic_r50_n8192"]   # 500 steps, as the workload defines
    t0 = time.perf_counter()
    X, T, plain_train = LR.collect_restarts(w, seeds=list(range(100, 164)), device=device)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, loss = LR.train_proposal(w.r, X, T, w.R, hidden=256, epochs=args.mlp_epochs, batch=256, lr=1e-3,
                                  seed=7, device=device)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    LR.run_filter(w, 5, "plain", device=device)          # warm-up
    rm_p, sps_p, rs_p = LR.run_filter(w, 5, "plain", device=device)
    rm_l, sps_l, rs_l = LR.run_filter(w, 5, "learned", net=net, device=device)
    out = {"metric": "RMSE and filter steps/s, learned vs plain restart", "value": round(sps_l, 3),
           "unit": "filter steps/s", "n_gpus": 1, "steps": w.steps, "warmup": 1, "ms_per_step": round(1e3 / sps_l, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
           "data": "synthetic (seeded Euler-Maruyama cubic sensor, scrambled Sobol nodes)",
           "config": {"workload": w.name, "r": w.r, "n": w.n, "steps": w.steps, "train_seeds": "100..163",
                      "eval_seed": 5, "mlp": f"{3 * w.r}-256-256-{2 * w.r} BF16", "epochs": args.mlp_epochs},
           "plain": {"rmse": rm_p, "steps_per_s": round(sps_p, 3), "restarts": rs_p},
           "learned": {"rmse": rm_l, "steps_per_s": round(sps_l, 3), "restarts": rs_l, "train_loss": loss},
           "training": {"rows": int(X.shape[0]), "collect_s": round(t_collect, 2), "train_s": round(t_train, 2),
                        "plain_rmse_train_mean": float(np.mean(plain_train))}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["batched_256"])
    ap.add_argument("--precision", default=None, choices=["bf16", "f32", "f32s", "f64"])
    ap.add_argument("--impl", default="yy", choices=["yy", "reference"])
    ap.add_argument("--fp32-steps", type=int, default=10, help="steps of the plain FP32 comparator")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--mlp-epochs", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-sublines", dest="sublines", action="store_false",
                    help="skip the r = 100, batched and large-scale sub-lines of the default workload")
    ap.add_argument("--shard", default="trajectories", choices=["trajectories", "rows"],
                    help="N > 1: independent trajectories per rank (default) or one filter's target rows split")
    ap.add_argument("--screen-type", default=None, choices=["bf16", "fp8"],
                    help="operands of the screen's Gram product (default: the workload's)")
    ap.add_argument("--screen-prefix", type=int, default=0,
                    help="BF16 screen: first-pass coordinate chunks of 64 (0 = chosen on the device)")
    ap.add_argument("--cta-pair", action="store_true",
                    help="BF16 screen on 2-CTA clusters (tcgen05.mma.cta_group::2); single CTAs by default")
    args = ap.parse_args()
    global CTA_PAIR
    CTA_PAIR = args.cta_pair
    if args.warmup < 3 and args.impl == "yy":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.shard == "rows":
        run_sharded(args)
    elif args.workload == "batched_256":
        run_batch(args)
    elif args.workload == "cubic_r50_n8192":
        run_learned(args)
    else:
        run_yy(args)


if __name__ == "__main__":
    main()
