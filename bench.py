#!/usr/bin/env python3
"""Throughput of the improved Yau--Yau filter's online stage on GB300.

One step = prediction (multi-scale kernel sum) + correction + normalisation + estimate
+ restart test (and a restart when it fires), for one trajectory of the workload.
Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision bf16|f32|f64] [--impl yy|reference]

Under torchrun (N > 1) every rank runs an independent trajectory of the same workload
(different seed); the path shards by trajectory with no collective, so the value is the
sum of trajectory-steps per second over ranks (weak scaling).  --impl reference times the
FP64 CPU oracle on a bounded sample of the same workload (rank 0 only).
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
# kernel, from one ncu capture of the workload (profiles/k_ksum_tc_cubic_r1000_n65536.md),
# keyed by workload and screen operands.  An entry is removed whenever the kernel changes
# after its capture.
NCU_TRAFFIC = {("cubic_r1000_n65536", "fp8"): 39.31392e6 + 0.466432e6}
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
    return flt


def _algorithmic_flops(w, precision, screen=None, stage=64):
    """Per prediction launch: BF16 path -> the Gram products the screen runs, i.e. per
    screened block of 128 targets x 256 sources 2 x 128 x 256 x (64 k) flops for the first
    pass over the first 64 k coordinates, plus 2 x 128 x 256 x r for every block screened
    again over all coordinates (screen = (k, blocks, rescreened); with the symmetric screen
    the blocks cover the upper block triangle, about half of the n^2 pairs);
    FP32/FP64 path -> difference form, 3 flops per coordinate per pair."""
    if precision == "bf16":
        k, tiles, resc = screen
        return 2.0 * 128 * 256 * (tiles * min(stage * k, w.r) + resc * w.r), "tensor"
    return 3.0 * w.n * w.n * w.r, "alu"


def _config(w, prec):
    return {"workload": w.name, "r": w.r, "n": w.n, "n_scales": w.n_scales, "dt": w.dt,
            "R": w.R, "restart_interval": w.restart_interval, "ess_frac": w.ess_frac,
            "precision": prec, "trajectories_per_gpu": 1, "time_loop": "one CUDA graph of K steps",
            "screen_operands": w.screen_type if prec == "bf16" else None,
            "l2": f"inputs larger than L2 (u is {w.n * w.r * 4 / 1e6:.0f} MB)"}


def _rmse(est, truth):
    K, r = truth.shape
    return float(np.sqrt(np.sum((est - truth) ** 2) / (K * r)))


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
    tr = simulate(w.model, w.r, W + K, w.dt, seed=seed)
    stream = torch.cuda.Stream(device)
    flt = _make_filter(w, prec, seed, device, stream, screen_prefix=args.screen_prefix,
                       screen_type=args.screen_type)
    dys = torch.tensor(tr.dy, dtype=torch.float64, device=device)
    hist = torch.zeros((K, 2 * w.r + 4), dtype=torch.float64, device=device)
    with torch.cuda.stream(stream):
        if W:
            flt.run_steps(dys[:W])
        # the K timed steps as one CUDA graph (captured, not executed, here)
        flt.graph_capture(dys[W:W + K], hist)
    torch.cuda.synchronize()
    # ---- device-resident timed region --------------------------------------------
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
    mean, var, ess, z = flt.estimate()
    # ---- dominant kernel: prediction launches timed alone on the filter's stream ----
    n_pred = max(3, min(20, K))
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    pe0.record(stream)
    for _ in range(n_pred):
        flt.predict()
    pe1.record(stream)
    torch.cuda.synchronize()
    pred_ms = pe0.elapsed_time(pe1) / n_pred
    screen = None
    if prec == "bf16":
        last, nxt, tiles, resc = flt.screen()
        stage = 128 if args.screen_type == "fp8" else 64
        screen = {"operands": args.screen_type, "first_pass_stages": last, "stage_coords": stage,
                  "stages": ((w.r + 63) // 64 * 64 + stage - 1) // stage, "tiles": tiles,
                  "rescreened": resc, "exact_pairs": flt.counters()[1]}
    flops, bound = _algorithmic_flops(w, prec, None if screen is None else (last, tiles, resc),
                                      128 if args.screen_type == "fp8" else 64)
    with torch.cuda.stream(stream):
        flt.update(dys[0])   # leave the handle in a consistent state
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
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    peaks, src = _peaks()
    steps_per_s = whole_job_rate(K, ws, t_max / 1e3)
    if bound == "tensor":
        # the prediction launches are timed back to back on their own (about 0.1 s), so the
        # burst figure is the matching denominator
        peak = peaks.get("bf16_tflops", 1900.0)
        achieved = flops / (pred_ms / 1e3) / 1e12
        peak_note = f"{src}: bf16_tflops (burst; prediction launches timed alone)"
        if args.screen_type == "fp8":   # FP8 dense rate = 2 x BF16 (4.5 / 2.25 PFLOP/s nominal)
            peak = 2.0 * peak
            peak_note = f"{src}: 2 x bf16_tflops (fp8 nominal ratio; burst; prediction launches timed alone)"
    else:
        # float32 FMA pipes: 152 SMs x 128 lanes x 2 flops x max SM clock
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        achieved = flops / (pred_ms / 1e3) / 1e12
        peak_note = "derived: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock"
    out = {
        "metric": METRIC,
        "value": round(steps_per_s, 4),
        "unit": "filter steps/s",
        "n_gpus": ws,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(t_max / K, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        # screen operands + float32 exact evaluation, log-sum-exp and update
        "dtype": {"bf16": ("fp8+f32" if args.screen_type == "fp8" else "bf16+f32"), "f32": "f32", "f64": "f64"}[prec],
        "data": "synthetic (seeded Euler-Maruyama cubic sensor, scrambled Sobol nodes)",
        "config": _config(w, prec),
        "pair_evals_per_s": round(steps_per_s * w.n_scales * w.n * w.n, 1),
        "rmse": rmse,
        "restarts": restarts,
        "clocks": clk.summary(),
        "e2e": {"value": round(e2e_val, 4), "unit": "filter steps/s",
                "h2d_bytes_per_step": 8 * w.r, "d2h_bytes_per_step": 8 * (2 * w.r + 2) + 56},
        "gpu_launches": int(launches),
        "screen": screen,
        "roofline": {"bound": bound, "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": NCU_TRAFFIC.get((w.name, args.screen_type)) if prec == "bf16" else None,
                     "kernel": "prediction (kernel sum)", "kernel_ms": round(pred_ms, 4),
                     "peak_source": peak_note},
    }
    if args.fp32_steps > 0 and prec == "bf16":
        S = min(args.fp32_steps, K)
        out["fp32_comparator"] = _time_precision(w, "f32", S, W, tr, device)
        out["fp32_comparator"]["rmse_mixed_same_steps"] = _rmse(est[:S], tr.x[W:W + S])
    if args.cpu_baseline and ws == 1:   # the oracle's baseline runs at N = 1 only
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def _time_precision(w, prec, steps, warmup, tr, device):
    """Steps/s and RMSE of another precision of the same path (the plain FP32 form) over
    the first `steps` timed steps of the same trajectory."""
    import torch
    stream = torch.cuda.Stream(device)
    flt = _make_filter(w, prec, w.seed, device, stream)
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


class OracleSample:
    """The FP64 oracle as it stands, set up once on the workload (nodes, prior state,
    prepared drift) and timed on this host's cores on a bounded sample: the prediction for a
    block of target rows against all n sources plus the O(n r) correction, scaled to one
    full step."""

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

    def step_rate(self, seconds: float):
        F, w = self.F, self.w
        rows = int(min(w.n, max(self.cores, self.cores * math.floor(seconds / (self.t_row * self.cores)))))
        t0 = time.perf_counter()
        F.predict(self.p, self.prep, self.st.logw, 0, rows, n_threads=self.cores)
        t_pred = time.perf_counter() - t0
        t0 = time.perf_counter()
        lw = F.log_likelihood(self.p, self.prep.x, self.dy) + self.st.logw
        lam, lh = F.normalise(lw)
        F.estimate(self.prep.x, lh)
        t_upd = time.perf_counter() - t0
        step_s = t_pred * (w.n / rows) + t_upd
        return {"value": round(1.0 / step_s, 6), "unit": "filter steps/s", "cores": self.cores,
                "kind": "oracle",
                "sample": f"prediction of {rows} of {w.n} target rows (all sources, {w.n_scales} scales) "
                          f"+ one full correction/estimate, scaled to one step; {t_pred + t_upd:.1f} s of CPU work"}


def cpu_baseline(w, seconds: float):
    return OracleSample(w).step_rate(seconds)


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
           "config": _config(w, prec),
           "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "sample": vals[-1]["sample"], "value": v},
           "e2e": {"value": v, "unit": "filter steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": round(time.perf_counter() - t0, 2)}
    print(json.dumps(out), flush=True)


def run_batch(args):
    """256 ragged trajectories (r in 10..200, n log-uniform in 2048..32768, half cubic, half
    linear-Gaussian) advanced as one batch; value = trajectory-steps per second."""
    import torch
    from paper_2509_16896_gb300 import binding
    rank, ws_, local, dist = _dist()
    device = f"cuda:{local}"
    torch.cuda.set_device(device)
    W, K = args.warmup, args.steps
    # untimed steps before the timed ones: at least 8, so that the autotuner routes on
    # posteriors that have spread out rather than on the prior
    S = max(W, 8)
    members = batched_workloads(256, seed=shard_seed(4, rank), steps=S + K)
    prec = args.precision or "bf16"
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
    # prediction alone
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(bt.stream)
    for _ in range(3):
        bt.predict()
    p1.record(bt.stream)
    torch.cuda.synchronize()
    pred_ms = p0.elapsed_time(p1) / 3
    h = hist.cpu().numpy()
    rm_c, rm_l = [], []
    for b, (m, t) in enumerate(zip(members, trs)):
        est = h[:, bt.hist_off[b]:bt.hist_off[b] + m.r]
        rm = _rmse(est, t.x[S:S + K])
        (rm_c if m.model == "cubic" else rm_l).append(rm)
    if rank != 0:
        return
    flops = float(sum(2.0 * m.n * m.n * m.r for m in members))
    peaks, src = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = flops / (pred_ms / 1e3) / 1e12
    out = {"metric": "trajectory-steps/s, 256 ragged filters in one batch",
           "value": round(whole_job_rate(256 * K, ws_, ms / 1e3), 2),
           "unit": "trajectory-steps/s", "n_gpus": ws_, "steps": K, "warmup": S, "ms_per_step": round(ms / K, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
           "data": "synthetic (seeded Euler-Maruyama cubic sensor / linear-Gaussian, scrambled Sobol nodes)",
           "config": {"workload": "batched_256", "trajectories": 256, "r": "10..200", "n": "2048..32768 log-uniform",
                      "n_scales": 2, "schedule": {"bn": bn, "grid": grid, "autotune_s": round(t_tune, 2),
                                                  "fp32_form_members": int(routing.sum()),
                                                  "fp32_form_max_r": int(max([m.r for m, p in zip(members, routing) if p] or [0]))},
                      "time_loop": "one CUDA graph of K batched steps"},
           "gpu_launches": int(launches), "clocks": clk.summary(),
           "rmse_cubic_mean": float(np.mean(rm_c)), "rmse_linear_mean": float(np.mean(rm_l)),
           "roofline": {"bound": "tensor", "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "kernel": "batched prediction (persistent)", "kernel_ms": round(pred_ms, 4)}}
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
    ap.add_argument("--precision", default=None, choices=["bf16", "f32", "f64"])
    ap.add_argument("--impl", default="yy", choices=["yy", "reference"])
    ap.add_argument("--fp32-steps", type=int, default=10, help="steps of the plain FP32 comparator")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--mlp-epochs", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--screen-type", default=None, choices=["bf16", "fp8"],
                    help="operands of the screen's Gram product (default: the workload's)")
    ap.add_argument("--screen-prefix", type=int, default=0,
                    help="BF16 screen: first-pass coordinate chunks of 64 (0 = chosen on the device)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "yy":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_256":
        run_batch(args)
    elif args.workload == "cubic_r50_n8192":
        run_learned(args)
    else:
        run_yy(args)


if __name__ == "__main__":
    main()
