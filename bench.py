#!/usr/bin/env python
"""Throughput benchmark of the detection path: strain-seconds analysed per second.

Default workload (the full-size configuration): one hour of seeded two-detector
2048 Hz coloured noise with 200 Newtonian chirps, Welch PSD epochs of 8 s with
a 64 s look-back, 1 s whitening FIR with a 32 Hz highpass, 1.5 s windows at a
16 Hz stride (57,600 windows), a ResNet34-style 1D network with GroupNorm(16)
and seeded weights, 1 s integration and 8 s clustering.  One step = one pass
of the whole path (PSD, filter build, whitening, windows, network,
integration, triggers) over that hour, inputs resident in HBM.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
Multi-GPU (torchrun): every rank analyses its own independent hour (weak
scaling, no data-path collective); the barrier and max-over-ranks timing use
torch.distributed.
"""
from __future__ import annotations

import argparse
import csv
import dataclasses
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2403_18661_gb300 import dist as pdist  # noqa: E402
from paper_2403_18661_gb300 import inputs  # noqa: E402

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2  # GB300: 1.25 TFLOP/s FP64 nominal = 152 SMs x 2 FMA/clk x 2 x 2.07 GHz


def n_sm() -> int:
    """Streaming multiprocessors of the current device (read from the device)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
    else:
        d = dict(FALLBACK_PEAKS)
        d["_source"] = "fallback"
    d["n_sm"] = n_sm()
    return d


def file_hash(rel: str) -> str:
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(kernel: str, algo_bytes_per_launch: float):
    """Per-launch DRAM bytes of `kernel`: the DRAM/algorithmic ratio of the committed
    ncu capture (profiles/traffic.json) times this run's algorithmic bytes per launch;
    None if there is no capture or its source file changed since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or file_hash(e["source"]) != e.get("src_sha256_16"):
        return None
    return e["dram_over_algorithmic"] * algo_bytes_per_launch


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = list(csv.reader(io.StringIO(self.tmp.read())))
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- oracle timing

def oracle_sample(wl, x: np.ndarray, w: np.ndarray, n_epochs: int, n_windows: int, seed: int = 0):
    """Time the FP64 oracle on a bounded sample of the workload and extrapolate to
    strain-seconds per second: PSD + filter + whitening of n_epochs epochs (both
    detectors) and the network on n_windows windows."""
    from oracle import oracle as orc
    rng = np.random.default_rng(seed)
    x64 = x.astype(np.float64)
    eps = sorted(rng.choice(wl.n_epochs, size=min(n_epochs, wl.n_epochs), replace=False).tolist())
    t0 = time.perf_counter()
    psd = orc.psd_epochs(x64, wl, eps)
    white = orc.whiten(x64, wl, psd, eps)
    t_white = time.perf_counter() - t0
    # windows that start inside the first sampled epoch's whitened span
    span = white.shape[1]
    n_fit = (span - wl.win_len) // wl.stride + 1
    n_w = min(n_windows, n_fit)
    t0 = time.perf_counter()
    orc.infer_windows(wl.net, w, white, wl.win_len, 0, wl.stride, n_w)
    t_net = time.perf_counter() - t0
    epoch_s = (wl.epoch_len if wl.epoch_len else wl.n_white) / wl.fs
    win_per_s = wl.fs / wl.stride
    sec_per_strain_s = t_white / (len(eps) * epoch_s) + t_net / n_w * win_per_s
    return {"value": 1.0 / sec_per_strain_s, "unit": "strain-s/s", "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"{len(eps)} PSD epochs (Welch + FP64 filter + direct FIR, 2 detectors) and {n_w} "
                      f"network windows, extrapolated per analysed second ({win_per_s:g} windows/s, "
                      f"{epoch_s:g} s epochs)",
            "seconds": t_white + t_net}


def workload_by_name(name: str, n_win: int = 0):
    if name == "hour":
        wl = inputs.HOUR_RESNET34
    elif name == "timeslides":
        return inputs.TIMESLIDE_DAY
    elif name == "plain64":
        wl = inputs.PLAIN_64S
    else:
        raise SystemExit(f"unknown workload {name}")
    if n_win:
        if wl.epoch_len == 0:
            raise SystemExit("--n-win applies to the epoch workloads")
        wl = dataclasses.replace(wl, n_win=n_win, n_chirps=max(1, wl.n_chirps * n_win // wl.n_win),
                                 name=f"{wl.name}-{n_win}win", duration_s=n_win * wl.stride / wl.fs)
    return wl


def dist_setup():
    return pdist.env()


def roofline_for(dom: dict, peaks: dict, step_ms_total: float) -> dict:
    """Roofline of the dominant kernel from its live CUDA-event time and algorithmic work."""
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    sms = peaks["n_sm"]
    name = dom["name"]
    if name.startswith("conv_gemm_fp32"):
        bound, unit = "alu", "TFLOP/s"
        achieved = dom["algo_flops"] / (dom["total_ms"] / 1000.0) / 1e12
        peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        src = f"derived: {sms} SMs (read from the device) x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 x {sm_max:g} MHz"
    elif name.startswith("filter_build_fp64"):
        bound, unit = "alu", "TFLOP/s"
        achieved = dom["algo_flops"] / (dom["total_ms"] / 1000.0) / 1e12
        peak = sms * FP64_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        src = f"derived: {sms} SMs (read from the device) x {FP64_LANES_PER_SM} FP64 FMA lanes x 2 x {sm_max:g} MHz"
    elif "bf16" in name:
        bound, unit = "tensor", "TFLOP/s"
        achieved = dom["algo_flops"] / (dom["total_ms"] / 1000.0) / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        src = f"{peaks['_source']} bf16_tflops_sustained"
    else:
        bound, unit = "hbm", "GB/s"
        achieved = dom["algo_bytes"] / (dom["total_ms"] / 1000.0) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        src = f"{peaks['_source']} hbm_gbs"
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "peak_source": src,
            "traffic": measured_traffic(name, dom["algo_bytes"] / max(dom["launches"], 1)),
            "launches": dom["launches"], "ms_per_launch": dom["total_ms"] / max(dom["timed"], 1),
            "share_of_step": dom["total_ms"] / max(step_ms_total, 1e-9)}


def tune_tiles(ctx, stream, n_win: int = 1024):
    """Autotune a BF16 context (set-up, outside every timed region): the conv tiles of a per-layer
    network, or the launch knobs of a fused one.  Returns a summary, or None where nothing is tunable."""
    from paper_2403_18661_gb300 import abi
    try:
        ctx.autotune(n_win, stream=stream)
    except abi.AfgError as e:
        if e.status == abi.AFG_ERR_UNSUPPORTED:
            return None
        raise
    try:
        tiles = ctx.tiles()
    except abi.AfgError as e:
        if e.status != abi.AFG_ERR_UNSUPPORTED:
            raise
        return {"n_win": n_win, "fused_tuning": ctx.fused_tuning()}  # fused network: no per-layer tiles
    return {"n_win": n_win, "layers": len(tiles),
            "sum_us_default": round(sum(t["us_default"] for t in tiles), 1),
            "sum_us_chosen": round(sum(t["us_chosen"] for t in tiles), 1),
            "chosen": sorted({(t["orient"], t["wpc"], t["kb"], t["stages"], t["acc_bufs"]) for t in tiles})}


def layer_roofline(tiles: list, n_win: int, conv_ms: float, peaks: dict) -> dict:
    """Per-layer roofline of the tensor-core convolutions: each layer's time bound is the larger of
    its algorithmic FLOPs at the sustained BF16 rate and its algorithmic bytes (input, residual and
    output once, plus weights) at the measured HBM rate; the network's bound is their sum.  frac =
    bound / measured conv time per step.  Layers whose FLOP/byte is below the ridge point are HBM-bound."""
    tf = peaks.get("bf16_tflops_sustained", 1700.0) * 1e12
    bw = peaks.get("hbm_gbs", 6800.0) * 1e9
    t_bound, t_hbm, n_hbm = 0.0, 0.0, 0
    for t in tiles:
        flops = 2.0 * n_win * t["lout"] * t["cout"] * t["taps"] * t["cin"]
        nbytes = 2.0 * n_win * ((t["lin"] + 2) * t["cin"] + (t["lout"] + 2) * t["cout"] * (2 if t["residual"] else 1)) \
            + 2.0 * t["taps"] * t["cin"] * t["cout"]
        tc, tm = flops / tf, nbytes / bw
        t_bound += max(tc, tm)
        if tm > tc:
            t_hbm += tm
            n_hbm += 1
    return {"bound_ms": t_bound * 1e3, "conv_ms": conv_ms, "frac": t_bound * 1e3 / max(conv_ms, 1e-9),
            "layers": len(tiles), "hbm_bound_layers": n_hbm, "hbm_bound_share_of_bound": t_hbm / max(t_bound, 1e-12),
            "ridge_flop_per_byte": tf / bw,
            "peaks": "measured bf16_tflops_sustained and hbm_gbs" if peaks.get("_source") != "fallback" else "fallback"}


def time_bf16_same_workload(wl, w, xd, args, stream, flush, peaks, world):
    """The same workload through the BF16 tensor-core network (context of its own),
    timed like the FP32 value; returned as a sub-result with the ratio to FP32."""
    import torch

    from paper_2403_18661_gb300 import abi
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    tiles = None if args.no_tune else tune_tiles(ctx, stream)
    out = None
    for _ in range(args.warmup):
        out = ctx.analyze(xd, trig_cap=65536, out=out)
    ctx.sync()
    ctx.profile_enable(True)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.analyze(xd, trig_cap=65536, out=out)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    kstats = ctx.profile_read()
    ctx.sync()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    value, _, job_s = pdist.job_throughput(wl.n_win * wl.stride / wl.fs * args.steps, total_ms / 1000.0, world)
    dom = max(kstats, key=lambda k: k["total_ms"])
    lroof = None
    try:
        geo = ctx.tiles()
    except abi.AfgError:
        geo = []
    if geo and dom["name"].startswith("conv_gemm_bf16"):
        lroof = layer_roofline(geo, wl.n_win, dom["total_ms"] / args.steps, peaks)
    ctx.close()
    return {"value": value, "unit": "strain-s/s", "ms_per_step": job_s * 1000.0 / args.steps, "dtype": "bf16",
            "roofline": roofline_for(dom, peaks, job_s * 1000.0), "layer_roofline": lroof,
            "gpu_launches": int(sum(k["launches"] for k in kstats)), "tiles": tiles}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    if args.workload == "resample":
        from oracle import oracle as orc
        fs_in, M, sec = 16384, 8, 20
        rng = np.random.default_rng(99)
        x = rng.standard_normal((2, sec * fs_in + 2 * 10 * M)) * 1e-21
        vals, total = [], 0.0
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            orc.resample(x, M)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                vals.append(sec / dt)
                total += dt
        value = statistics.mean(vals)
        samp = f"{sec} s of two-detector 16384 Hz strain decimated by 8 per step (FP64 oracle, numpy)"
        print(json.dumps({"metric": "strain-seconds/s resampled 16384 -> 2048 Hz", "impl": "reference", "value": value,
                          "unit": "strain-s/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "1h-2det-16384Hz-decimate8"},
                          "cpu_baseline": {"value": value, "unit": "strain-s/s", "cores": 1, "kind": "oracle",
                                           "sample": samp},
                          "e2e": {"value": value, "unit": "strain-s/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    if args.workload == "whiten":
        wl = whiten_workload(args.n_win)
        wl_s = dataclasses.replace(wl, n_win=(160 * wl.epoch_len) // wl.stride)
        x, _ = inputs.make_strain(wl_s)
        vals, total = [], 0.0
        for i in range(args.warmup + args.steps):
            r = oracle_whiten_sample(wl_s, x, n_epochs=128, seed=i)
            if i >= args.warmup:
                vals.append(r["value"])
                total += r["seconds"]
        value = statistics.mean(vals)
        print(json.dumps({"metric": "strain-seconds/s Welch+filter+whitening", "impl": "reference", "value": value,
                          "unit": "strain-s/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": wl.name, "analysed_s": wl.n_white / wl.fs},
                          "cpu_baseline": {"value": value, "unit": "strain-s/s", "cores": r["cores"],
                                           "kind": "oracle", "sample": r["sample"]},
                          "e2e": {"value": value, "unit": "strain-s/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    wl = workload_by_name(args.workload, args.n_win)
    x, _ = inputs.make_strain(wl)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    vals, total = [], 0.0
    for i in range(args.warmup + args.steps):
        r = oracle_sample(wl, x, w, n_epochs=1, n_windows=args.ref_windows, seed=i)
        if i >= args.warmup:
            vals.append(r["value"])
            total += r["seconds"]
    value = statistics.mean(vals)
    out = {"metric": "strain-seconds/s whiten+ResNet", "impl": "reference", "value": value, "unit": "strain-s/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "windows": wl.n_win, "seconds": wl.duration_s},
           "cpu_baseline": {"value": value, "unit": "strain-s/s", "cores": r["cores"], "kind": "oracle",
                            "sample": r["sample"]},
           "e2e": {"value": value, "unit": "strain-s/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2403_18661_gb300 import abi

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = workload_by_name(args.workload, args.n_win)
    # each rank analyses its own hour of strain (weak scaling)
    wl_r = dataclasses.replace(wl, seed=pdist.rank_seed(wl.seed, rank)) if rank else wl
    x, _ = inputs.make_strain(wl_r)
    w = inputs.make_weights(wl.net, wl.weight_seed)
    precision = abi.AFG_BF16 if args.precision == "bf16" else abi.AFG_FP32
    ctx = abi.Context(wl, w, precision=precision)
    xd = torch.from_numpy(x).to(dev)
    tiles = tune_tiles(ctx, torch.cuda.current_stream()) if precision == abi.AFG_BF16 and not args.no_tune else None
    trig_cap = 65536
    out = (torch.empty(wl.n_win, dtype=torch.float32, device=dev),
           torch.empty(wl.n_win - wl.n_int + 1, dtype=torch.float32, device=dev),
           torch.empty(trig_cap, dtype=torch.int64, device=dev),
           torch.zeros(1, dtype=torch.int64, device=dev))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.analyze(xd, trig_cap=trig_cap, out=out)
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    ctx.profile_enable(True)
    step_ms = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the step's events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.analyze(xd, trig_cap=trig_cap, out=out)
        e1.record(stream)
        step_ms.append((e0, e1))
    barrier()
    ctx.profile_enable(False)
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in step_ms]
    total_ms = sum(step_ms)
    kstats = ctx.profile_read()
    seconds_per_step = wl.n_win * wl.stride / wl.fs
    value, _, job_s = pdist.job_throughput(seconds_per_step * args.steps, total_ms / 1000.0, world)
    total_ms = job_s * 1000.0

    # end to end through the public host-buffer call: H2D of the strain, D2H of statistic + triggers
    e2e = None
    if not args.no_e2e:
        xp = torch.from_numpy(x).pin_memory()
        stat_h = torch.empty(wl.n_win - wl.n_int + 1, dtype=torch.float32).pin_memory()
        trig_h = torch.empty(trig_cap, dtype=torch.int64).pin_memory()
        ctx.analyze_host(xp, trig_cap=trig_cap, stat_out=stat_h, trig_out=trig_h)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.analyze_host(xp, trig_cap=trig_cap, stat_out=stat_h, trig_out=trig_h)
        barrier()
        dt = time.perf_counter() - t0
        e2e_value, _, _ = pdist.job_throughput(seconds_per_step * args.steps, dt, world)
        e2e = {"value": e2e_value, "unit": "strain-s/s",
               "h2d_bytes_per_step": int(x.nbytes),
               "d2h_bytes_per_step": int(stat_h.numel() * 4 + 8 + trig_cap * 8)}

    peaks = load_peaks()
    bf16 = None  # same workload through the BF16 tensor-core network (every rank: it reduces across ranks)
    if precision == abi.AFG_FP32 and not args.no_bf16 and wl.net == inputs.RESNET34_NET:
        bf16 = time_bf16_same_workload(wl, w, xd, args, stream, flush, peaks, world)
        bf16["ratio_vs_fp32"] = bf16["value"] / value
    nested = args.workload == "hour" and not args.n_win
    del xd, flush
    torch.cuda.empty_cache()
    # the batching workload (every rank analyses its own day: weak scaling) and the serving workload
    # (one GPU), each with its own timing, nested in this line
    batched = bf16_batched_subresult(world, rank, local, peaks) if nested and not args.no_batched else None
    serving = None
    if nested and not args.no_serving and world == 1:
        serving = serving_measure(args.n_streams, 20.0, local)
        serving = {k: serving[k] for k in ("value", "unit", "latency_ms", "config", "windows_per_s", "roofline",
                                           "gpu_launches", "clocks", "e2e")}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    launches = int(sum(k["launches"] for k in kstats))
    dom = max(kstats, key=lambda k: k["total_ms"])
    roofline = roofline_for(dom, peaks, total_ms)
    kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3),
                           "share": round(k["total_ms"] / max(sum(q["total_ms"] for q in kstats), 1e-9), 4)}
               for k in kstats}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_sample(wl, x, w, n_epochs=2, n_windows=args.ref_windows)
        cpu.pop("seconds", None)

    out = {"metric": "strain-seconds/s whiten+ResNet", "value": value, "unit": "strain-s/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if precision == abi.AFG_FP32 else "bf16", "data": "synthetic",
           "config": {"workload": wl.name, "windows": wl.n_win, "analysed_s": seconds_per_step,
                      "net": "resnet34-1d-gn16" if wl.net == inputs.RESNET34_NET else "tiny-1d-gn8",
                      "precision": args.precision, "l2": "flushed between steps (512 MiB write)"},
           "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "bf16": bf16, "bf16_batched": batched, "serving": serving, "tiles": tiles,
           "clocks": clocks, "kernels": kernels}
    out["config"]["n_sm"] = peaks["n_sm"]
    print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def timeslide_measure(precision, n_seg, n_shift, steps, warmup, world, rank, local, with_far=True, clocks=True,
                      shard=False):
    """Time `steps` steps of the timeslide background (segments x timeslides through
    afg_batch_run, replayed as one CUDA graph, then the FAR of the background triggers)
    after `warmup` untimed steps.  Returns the measurement (every rank) and, on rank 0, the
    per-kernel shares of one direct (profiled) call.

    shard (world > 1): one background split across the ranks.  Every rank holds the same
    segments and takes a contiguous range of the timeslides; each step ends with the
    background triggers of all ranks gathered (each rank's sorted by the library's FAR sort,
    then two NCCL all_gathers of counts and values) and the FAR assigned against the whole
    background.  Otherwise every rank analyses its own day (independent work)."""
    import torch

    from paper_2403_18661_gb300 import abi

    dev = torch.device("cuda", torch.cuda.current_device())
    wl = inputs.TIMESLIDE_DAY
    shard = shard and world > 1
    k_first, n_k = pdist.shift_range(n_shift, world, rank) if shard else (1, n_shift)
    lengths = inputs.segment_lengths(n_seg=40, total_s=86400)[:n_seg]
    seed = wl.seed if shard else pdist.rank_seed(wl.seed, rank)  # sharded: the same strain on every rank
    x, segs = inputs.make_segments(lengths, seed=seed, chirp_every_s=300.0, workers=min(16, os.cpu_count() or 1))
    w = inputs.make_weights(wl.net, wl.weight_seed)
    ctx = abi.Context(wl, w, precision=precision)
    xd = torch.from_numpy(x).to(dev)
    del x
    n_win, tw, ts = ctx.batch_layout(segs, n_k, wl.fs, k_first)
    livetime = tw * wl.stride / wl.fs  # background seconds this rank analyses per step
    livetime_all = pdist.sum_over_ranks(livetime, world) if shard else livetime
    stream = torch.cuda.Stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = None
    trig_cap = 1 << 20
    far_out = None
    local_out = None

    def far_step():
        nonlocal local_out
        logits, stat, trig, n_trig = out
        if not shard:
            return ctx.far(stat, stat[:1024], livetime, bg_idx=trig, n_bg=n_trig, bg_cap=trig_cap, out=far_out,
                           stream=stream)
        # this rank's background sorted on the device, all ranks' gathered, then the FAR of this
        # rank's foreground against the whole background
        local_out = ctx.far(stat, stat[:0], livetime, bg_idx=trig, n_bg=n_trig, bg_cap=trig_cap, out=local_out,
                            stream=stream)
        stream.synchronize()
        n_local = min(int(n_trig.item()), trig_cap)
        bg_all = pdist.gather_background(local_out[2][:n_local].contiguous(), world)
        return ctx.far(bg_all, stat[:1024], livetime_all, stream=stream)

    tuning = None
    if precision == abi.AFG_BF16:  # the fused network's knobs, tuned before anything is timed
        try:
            ctx.autotune(4096, stream=stream)
            tuning = ctx.fused_tuning()
        except abi.AfgError as e:
            if e.status != abi.AFG_ERR_UNSUPPORTED:
                raise
    with torch.cuda.stream(stream):
        # one direct call with per-kernel timing for the shares, then the captured graph
        ctx.profile_enable(True)
        out = ctx.batch_run(xd, segs, n_k, wl.fs, trig_cap=trig_cap, out=out, stream=stream, shift_first=k_first)
        if with_far:
            far_out = far_step()
        kstats = ctx.profile_read()
        for _ in range(warmup):
            out = ctx.batch_run(xd, segs, n_k, wl.fs, trig_cap=trig_cap, use_graph=True, out=out, stream=stream,
                                shift_first=k_first)
            if with_far:
                far_out = far_step()
    pdist.barrier(world)
    sampler = ClockSampler(local) if (rank == 0 and clocks) else None
    if sampler:
        sampler.start()
    ctx.profile_enable(False)
    evs = []
    pdist.barrier(world)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.batch_run(xd, segs, n_k, wl.fs, trig_cap=trig_cap, use_graph=True, out=out, stream=stream,
                          shift_first=k_first)
            if with_far:
                far_out = far_step()
            e1.record(stream)
            evs.append((e0, e1))
    pdist.barrier(world)
    ctx.sync(stream)
    clk = sampler.stop() if sampler else None
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    n_bg = int(out[3].item())
    far_min = float(far_out[1][:1024].min().item()) if (with_far and n_bg) else None
    value, _, job_s = pdist.job_throughput(livetime * steps, total_ms / 1000.0, world)
    ctx.close()
    del xd, flush
    return {"value": value, "ms_per_step": job_s * 1000.0 / steps, "livetime_s": livetime_all, "windows": tw,
            "segments": len(segs), "strain_s": int(sum(lengths)), "timeslides": n_shift, "background_triggers": n_bg,
            "far_min_per_s": far_min, "kstats": kstats, "clocks": clk, "steps": steps, "warmup": warmup,
            "sharded": shard, "shift_range": [k_first, n_k], "tuning": tuning}


def timeslide_summary(m, peaks, precision):
    """Roofline and kernel shares of a timeslide measurement (rank 0)."""
    kstats = m["kstats"]
    dom = max(kstats, key=lambda k: k["total_ms"])
    launches_per_step = int(sum(k["launches"] for k in kstats))
    return {"value": m["value"], "unit": "strain-s/s", "ms_per_step": m["ms_per_step"], "steps": m["steps"],
            "warmup": m["warmup"], "dtype": "bf16" if precision else "f32",
            "config": {"workload": inputs.TIMESLIDE_DAY.name if m["segments"] == 40 and m["timeslides"] == 100
                       else f"timeslides-{m['segments']}seg-{m['timeslides']}shifts-tiny-4Hz",
                       "segments": m["segments"], "strain_s": m["strain_s"], "timeslides": m["timeslides"],
                       "windows": m["windows"], "livetime_s": m["livetime_s"],
                       "graph": "one CUDA graph per step + the FAR sort", "l2": "flushed between steps (512 MiB write)",
                       "background_triggers": m["background_triggers"], "far_min_per_s": m["far_min_per_s"]},
            "roofline": roofline_for(dom, peaks, sum(k["total_ms"] for k in kstats)),
            "gpu_launches": launches_per_step * m["steps"], "clocks": m["clocks"],
            "fused_tuning": m["tuning"],
            "kernels_direct_call": {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3)}
                                    for k in kstats}}


def bf16_batched_subresult(world, rank, local, peaks):
    """The batching workload (40 uneven segments, about 1 day, 100 timeslides, the 16-channel
    network in BF16, one graph per step), plus the BF16 / FP32 ratio measured on a subset
    (4 segments x 10 timeslides) that the FP32 path finishes in well under a second per step."""
    from paper_2403_18661_gb300 import abi
    full = timeslide_measure(abi.AFG_BF16, 40, 100, 3, 3, world, rank, local)
    sub16 = timeslide_measure(abi.AFG_BF16, 4, 10, 5, 3, world, rank, local, clocks=False)
    sub32 = timeslide_measure(abi.AFG_FP32, 4, 10, 5, 3, world, rank, local, clocks=False)
    if rank != 0:
        return None
    r = timeslide_summary(full, peaks, abi.AFG_BF16)
    r["vs_fp32_subset"] = {"segments": 4, "timeslides": 10, "windows": sub16["windows"],
                           "bf16": sub16["value"], "fp32": sub32["value"], "ratio": sub16["value"] / sub32["value"]}
    return r


def run_timeslides(args):
    """One step = the whole timeslide background of ~1 day: whitening of every
    segment, every window of every (segment, timeslide) series through the
    network in one persistent launch, integration and clustering of every
    series (replayed as one CUDA graph), then the false-alarm rates: the
    background triggers sorted on the device and ranked against 1024
    statistic samples."""
    import torch
    import torch.distributed as dist

    from paper_2403_18661_gb300 import abi

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    precision = abi.AFG_BF16 if args.precision == "bf16" else abi.AFG_FP32
    m = timeslide_measure(precision, args.n_seg, args.n_shift, args.steps, args.warmup, world, rank, local,
                          shard=True)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    r = timeslide_summary(m, load_peaks(), precision)
    res = {"metric": "strain-seconds/s whiten+ResNet (timeslide background livetime)", "value": r["value"],
           "unit": "strain-s/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "strong" if m["sharded"] else "weak",
           "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic", "config": r["config"],
           "roofline": r["roofline"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
           "fused_tuning": r["fused_tuning"], "kernels_direct_call": r["kernels_direct_call"]}
    print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def serving_measure(n_streams, serve_seconds, local):
    """Continuous-batching serving of n streams of 0.25 s chunks (rank 0 only; returns the result).

    Phase 1 (not timed) fills every stream past its 64 s PSD look-back.
    Phase 2 (latency) pushes chunks with Poisson arrivals at 4 per second per
    stream for >= 9191 pushes and reports p50/p99 push-to-statistic latency.
    Phase 3 (throughput) pushes the rest as fast as the host can and reports
    the aggregate strain-seconds analysed per second of wall time."""
    import heapq

    import torch

    from paper_2403_18661_gb300 import abi

    wl = inputs.SERVING_128
    chunk = 512
    warm_s, lat_s, thr_s = 66.0, max(1.0, 9300 / (4.0 * n_streams)), serve_seconds
    total_s = warm_s + lat_s * 1.6 + thr_s + 2.0
    n_tot = int(total_s * wl.fs)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        xs = list(ex.map(lambda i: np.stack([inputs.coloured_noise(n_tot, wl.seed * 1000 + 2 * i + d)
                                             for d in range(2)]).astype(np.float32), range(n_streams)))
    w = inputs.make_weights(wl.net, wl.weight_seed)
    ctx = abi.Context(wl, w, precision=abi.AFG_BF16)
    ctx.stream_start(max_streams=n_streams, max_chunk=4096)
    sids = [ctx.stream_open() for _ in range(n_streams)]
    pos = [0] * n_streams
    n_warm = int(warm_s * wl.fs)
    for i, sid in enumerate(sids):
        for a in range(0, n_warm, 4096):
            ctx.stream_push(sid, xs[i][:, a:a + 4096])
        pos[i] = n_warm
    ctx.stream_flush(120.0)
    for sid in sids:
        ctx.stream_poll(sid)
    # phase 2: Poisson arrivals, real time
    rng = np.random.default_rng(11)

    def poisson_phase(min_pushes, min_s):
        t0 = time.perf_counter()
        heap = [(float(rng.exponential(0.25)), i) for i in range(n_streams)]
        heapq.heapify(heap)
        n = 0
        while n < min_pushes or heap[0][0] < min_s:
            t_next, i = heapq.heappop(heap)
            dt = t0 + t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ctx.stream_push(sids[i], xs[i][:, pos[i]:pos[i] + chunk])
            pos[i] += chunk
            n += 1
            heapq.heappush(heap, (t_next + float(rng.exponential(0.25)), i))
            if pos[i] + chunk > n_tot - int(thr_s * wl.fs):
                break
        ctx.stream_flush(120.0)
        out = []
        for sid in sids:
            r = ctx.stream_poll(sid)
            out.append(r["t_done"] - r["t_push"])
        return n, np.concatenate(out) * 1000.0

    sampler = ClockSampler(local)
    sampler.start()
    pushes, lat = poisson_phase(9191, lat_s)
    # a short profiled Poisson phase (events around every launch; not used for the percentiles):
    # what one latency-phase step is made of
    ctx.profile_enable(True)
    st0 = ctx.stream_stats()
    n_prof, _ = poisson_phase(1024, 0.0)
    st1 = ctx.stream_stats()
    ctx.profile_enable(False)
    prof_steps = max(1, int(st1["steps"] - st0["steps"]))
    lat_kernels = {k["name"]: {"launches_per_step": round(k["launches"] / prof_steps, 3),
                               "us_per_launch": round(1000.0 * k["total_ms"] / max(k["timed"], 1), 2)}
                   for k in ctx.profile_read()}
    # phase 3: maximum offered load (the engine is idle here: counters start clean)
    n_thr = int(thr_s * wl.fs)
    # each round's 0.25 s chunks of every stream arrive as one burst (afg_stream_push_many): one
    # Python call per push would bound the offered load at the host (about 4.8 us per push); the
    # bursts are the client's arrays, assembled before the timed phase
    bursts = [np.stack([xs[i][:, pos[i] + a:pos[i] + a + chunk] for i in range(n_streams)])
              for a in range(0, n_thr, chunk)]
    ctx.profile_enable(True)
    stats0 = ctx.stream_stats()
    t1 = time.perf_counter()
    pushed_samples = 0
    for burst in bursts:
        ctx.stream_push_many(sids, burst)
        pushed_samples += chunk * n_streams
    ctx.stream_flush(300.0)
    wall = time.perf_counter() - t1
    clocks = sampler.stop()
    stats1 = ctx.stream_stats()
    ctx.profile_enable(False)
    kstats = ctx.profile_read()
    for sid in sids:
        ctx.stream_poll(sid)
    value = pushed_samples / wl.fs / wall
    n_steps = max(1, int(stats1["steps"] - stats0["steps"]))
    n_results = int(stats1["windows"] - stats0["windows"])
    dom = max(kstats, key=lambda k: k["total_ms"]) if kstats else None
    out = {"metric": "strain-seconds/s whiten+ResNet (serving, continuous batching)", "value": value,
           "unit": "strain-s/s", "n_gpus": 1, "steps": int(stats1["steps"] - stats0["steps"]), "warmup": 0,
           "ms_per_step": 1000.0 * wall / max(1, stats1["steps"] - stats0["steps"]), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": wl.name, "streams": n_streams, "chunk_samples": chunk,
                      "arrivals": "Poisson, 4 pushes/s per stream (latency phase); one burst of every "
                                  "stream's next chunk per afg_stream_push_many call (throughput phase)",
                      "latency_pushes": pushes,
                      "throughput_seconds_per_stream": thr_s},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                          "p99": float(np.percentile(lat, 99)), "results": int(lat.size)},
           "latency_step_kernels": {"pushes": n_prof, "steps": prof_steps, "kernels": lat_kernels},
           "windows_per_s": n_results / wall, "clocks": clocks,
           "roofline": roofline_for(dom, load_peaks(), sum(k["total_ms"] for k in kstats)) if dom else None,
           "gpu_launches": int(sum(k["launches"] for k in kstats)),
           "kernels": {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3)} for k in kstats},
           "e2e": {"value": value, "unit": "strain-s/s",
                   "h2d_bytes_per_step": int(pushed_samples * 2 * 4 / n_steps),
                   "d2h_bytes_per_step": int(n_results * 32 / n_steps),
                   "note": "wall time from the first host push to the last result on the host (pinned staging "
                           "copies in, 32-byte results out)"}}
    ctx.close()
    return out


def run_serving(args):
    import torch
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    torch.cuda.set_device(0)
    print(json.dumps(serving_measure(args.n_streams, args.serve_seconds, local)), flush=True)
    return 0


def whiten_workload(n_win: int = 0):
    """Six hours of seeded two-detector coloured noise in epoch mode: the Welch PSD of the
    64 s before every 8 s epoch, its FP64 filter and the overlap-save whitening (Sec. IV ("Noise sampling"),
    Sec. VI).  Windows only size the whitened span (16 Hz, as the 1 h workload)."""
    base = inputs.HOUR_RESNET34
    n = n_win or 6 * base.n_win
    return dataclasses.replace(base, name=f"{n * base.stride // base.fs // 3600}h-2det-welch-filter-whiten"
                               if not n_win else f"welch-filter-whiten-{n}win", n_win=n,
                               duration_s=n * base.stride / base.fs, n_chirps=0, seed=9876)


def oracle_whiten_sample(wl, x: np.ndarray, n_epochs: int, seed: int = 0):
    """The FP64 oracle's Welch + filter + direct-FIR whitening on n_epochs consecutive epochs of
    both detectors, starting at a seeded random epoch, extrapolated to strain-seconds per second."""
    from oracle import oracle as orc
    e0 = int(np.random.default_rng(seed).integers(0, max(wl.n_epochs - n_epochs, 0) + 1))
    lo = e0 * wl.epoch_len
    xs = x[:, lo:lo + wl.psd_len + n_epochs * wl.epoch_len + wl.crop].astype(np.float64)
    eps = list(range(n_epochs))  # epochs e0.. of x are epochs 0.. of xs
    t0 = time.perf_counter()
    psd = orc.psd_epochs(xs, wl, eps)
    orc.whiten(xs, wl, psd, eps)
    dt = time.perf_counter() - t0
    return {"value": n_epochs * wl.epoch_len / wl.fs / dt, "unit": "strain-s/s", "cores": orc.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"{n_epochs} consecutive epochs of 8 s (Welch of the 64 s before each, FP64 filter, direct "
                      f"2047-tap FIR, 2 detectors), extrapolated per analysed second"}


def run_whiten(args):
    """One step = steps a1-a3 over six hours: Welch periodograms and epoch means, FP64 filter
    build, overlap-save whitening of both detectors, device buffers resident (inputs and
    outputs, 355 MB each, exceed the 129 MB L2); e2e adds the host copies of the raw strain and
    of the whitened result."""
    import torch
    import torch.distributed as dist

    from paper_2403_18661_gb300 import abi

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = whiten_workload(args.n_win)
    wl_r = dataclasses.replace(wl, seed=pdist.rank_seed(wl.seed, rank)) if rank else wl
    x, _ = inputs.make_strain(wl_r)
    ctx = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    xd = torch.from_numpy(x).to(dev)
    n_psd, n_out = wl.n_epochs, wl.n_white
    psd = torch.empty((2, n_psd, wl.nfft // 2 + 1), dtype=torch.float64, device=dev)
    y = torch.empty((2, n_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctx.psd_estimate(xd, n_psd=n_psd, psd_step=wl.epoch_len, psd_span=wl.psd_len, out=psd)
        ctx.whiten(xd, psd, wl.psd_len, n_out, epoch_len=wl.epoch_len, out=y)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    big = x.nbytes > (129 << 20)
    flush = None if big else torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    ctx.profile_enable(True)
    evs = []
    barrier()
    for _ in range(args.steps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    ctx.profile_enable(False)
    clocks = sampler.stop() if sampler else None
    kstats = ctx.profile_read()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    sec = n_out / wl.fs
    value, _, job_s = pdist.job_throughput(sec * args.steps, total_ms / 1000.0, world)
    e2e = None
    if not args.no_e2e:
        xp = torch.from_numpy(x).pin_memory()
        yh = torch.empty((2, n_out), dtype=torch.float32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            xd.copy_(xp, non_blocking=True)
            step()
            yh.copy_(y, non_blocking=True)
            stream.synchronize()
        barrier()
        e2e_v, _, _ = pdist.job_throughput(sec * args.steps, time.perf_counter() - t0, world)
        e2e = {"value": e2e_v, "unit": "strain-s/s", "h2d_bytes_per_step": int(x.nbytes),
               "d2h_bytes_per_step": int(yh.numel() * 4)}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_whiten_sample(wl, x, n_epochs=128)
        cpu.pop("seconds")
    peaks = load_peaks()
    # the dominant kernel of the step (the FP64 filter build, ALU-bound); the HBM-bound FP32 kernels carry
    # their own rooflines in "kernels"
    dom = max((k for k in kstats if k["launches"]), key=lambda k: k["total_ms"])
    per_kernel = {k["name"]: roofline_for(k, peaks, job_s * 1000.0) for k in kstats if k["launches"]}
    out = {"metric": "strain-seconds/s Welch+filter+whitening", "value": value, "unit": "strain-s/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": job_s * 1000.0 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl.name, "analysed_s": sec, "epochs": n_psd, "n_raw": wl.n_raw,
                      "l2": "inputs larger than L2" if big else "flushed between steps (512 MiB write)"},
           "roofline": roofline_for(dom, peaks, job_s * 1000.0), "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(sum(k["launches"] for k in kstats)), "clocks": clocks, "kernels": per_kernel}
    print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_resample(args):
    """One step = decimation of 1 h of two-detector strain from 16384 Hz to 2048 Hz (Sec. IV.A),
    device buffers resident; e2e adds the host copies of the raw strain and of the result."""
    import torch
    import torch.distributed as dist

    from paper_2403_18661_gb300 import abi

    world, rank, local = dist_setup()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    fs_in, M, dur = 16384, 8, 3600.0
    n_in = int(fs_in * dur) + 2 * 10 * M  # the hour plus the filter's half-length at each end
    rng = np.random.default_rng(pdist.rank_seed(99, rank))
    x = (rng.standard_normal((2, n_in), dtype=np.float32) * np.float32(1e-21))
    wl = inputs.PLAIN_64S
    ctx = abi.Context(wl, inputs.make_weights(wl.net, wl.weight_seed))
    xd = torch.from_numpy(x).to(dev)
    n_out, first = abi.resample_size(n_in, M)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        y, _ = ctx.resample(xd, M)
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    ctx.profile_enable(True)
    evs = []
    barrier()
    for _ in range(args.steps):  # inputs (472 MB) exceed the 129 MB L2: no flush needed
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y, _ = ctx.resample(xd, M)
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    ctx.profile_enable(False)
    clocks = sampler.stop() if sampler else None
    kstats = ctx.profile_read()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    value, _, job_s = pdist.job_throughput(dur * args.steps, total_ms / 1000.0, world)
    e2e = None
    if not args.no_e2e:
        xp = torch.from_numpy(x).pin_memory()
        yh = torch.empty((2, n_out), dtype=torch.float32).pin_memory()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            xd.copy_(xp, non_blocking=True)
            y, _ = ctx.resample(xd, M)
            yh.copy_(y, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        barrier()
        e2e_v, _, _ = pdist.job_throughput(dur * args.steps, time.perf_counter() - t0, world)
        e2e = {"value": e2e_v, "unit": "strain-s/s", "h2d_bytes_per_step": int(x.nbytes),
               "d2h_bytes_per_step": int(yh.numel() * 4)}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        from oracle import oracle as orc
        sec = 60
        t0 = time.perf_counter()
        orc.resample(x[:, : sec * fs_in + 2 * 10 * M].astype(np.float64), M)
        dt = time.perf_counter() - t0
        cpu = {"value": sec / dt, "unit": "strain-s/s", "cores": 1, "kind": "oracle",
               "sample": f"{sec} s of two-detector 16384 Hz strain decimated by the FP64 oracle (numpy)"}
    peaks = load_peaks()
    dom = max(kstats, key=lambda k: k["total_ms"])
    out = {"metric": "strain-seconds/s resampled 16384 -> 2048 Hz", "value": value, "unit": "strain-s/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": job_s * 1000.0 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "1h-2det-16384Hz-decimate8", "n_in": n_in, "n_out": n_out, "taps": 2 * 10 * M + 1,
                      "l2": "inputs (472 MB) larger than L2"},
           "roofline": roofline_for(dom, peaks, job_s * 1000.0), "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(sum(k["launches"] for k in kstats)), "clocks": clocks}
    print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_rates(args):
    """Inference-rate sweep (Sec. IX: throughput vs inference rate; the online mode evaluates a
    window at every sample).  One step = the whole path (PSD epochs, whitening, every window through
    the paper's 16-channel network on tcgen05, integration, clustering) over 1 h of strain at a given
    rate; the line's value is the paper's 4 Hz rate, the sweep holds 1..64 Hz and 2048 Hz."""
    import torch

    from paper_2403_18661_gb300 import abi

    world, rank, local = dist_setup()
    if world > 1:
        raise SystemExit("the rate sweep runs on one GPU")
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = dataclasses.replace(inputs.HOUR_RESNET34, name="1h-tiny-rates", net=inputs.TINY_NET, stride=512,
                               n_win=3600 * 4, n_chirps=200)
    x, _ = inputs.make_strain(base)
    xd = torch.from_numpy(x).to(dev)
    w = inputs.make_weights(base.net, base.weight_seed)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    rates = [1, 2, 4, 8, 16, 32, 64, 2048]
    sweep, kst4, clocks = {}, None, None
    for r in rates:
        wl = dataclasses.replace(base, name=f"1h-tiny-{r}Hz", stride=2048 // r, n_win=3600 * r)
        assert wl.n_raw == base.n_raw
        res = {}
        for prec in (["bf16", "fp32"] if (r <= 64 and not args.no_fp32) else ["bf16"]):
            ctx = abi.Context(wl, w, precision=abi.AFG_BF16 if prec == "bf16" else abi.AFG_FP32)
            steps = args.steps if r < 2048 or prec == "bf16" else 1
            out = None
            for _ in range(args.warmup):
                out = ctx.analyze(xd, trig_cap=1 << 16, out=out)
            torch.cuda.synchronize()
            sampler = ClockSampler(0) if (r == 4 and prec == "bf16") else None
            if sampler:
                sampler.start()
                ctx.profile_enable(True)
            evs = []
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.analyze(xd, trig_cap=1 << 16, out=out)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            if sampler:
                ctx.profile_enable(False)
                clocks = sampler.stop()
                kst4 = ctx.profile_read()
            ctx.sync()
            ms = sum(a.elapsed_time(b) for a, b in evs) / steps
            res[prec] = {"strain_s_per_s": 3600.0 / (ms / 1000.0), "windows_per_s": wl.n_win / (ms / 1000.0),
                         "ms_per_step": ms}
            ctx.close()
        if "fp32" in res:
            res["bf16_over_fp32"] = res["bf16"]["strain_s_per_s"] / res["fp32"]["strain_s_per_s"]
        sweep[f"{r}Hz"] = res
    peaks = load_peaks()
    dom = max(kst4, key=lambda k: k["total_ms"])
    v4 = sweep["4Hz"]["bf16"]
    out = {"metric": "strain-seconds/s whiten+ResNet vs inference rate (tiny network, BF16)",
           "value": v4["strain_s_per_s"], "unit": "strain-s/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v4["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": "1h-tiny-rate-sweep", "rates_hz": rates, "value_at": "4 Hz",
                      "l2": "flushed between steps (512 MiB write)"},
           "roofline": roofline_for(dom, peaks, sum(k["total_ms"] for k in kst4)),
           "gpu_launches": int(sum(k["launches"] for k in kst4)), "clocks": clocks, "sweep": sweep}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="hour",
                    choices=["hour", "plain64", "timeslides", "serving", "resample", "rates", "whiten"])
    ap.add_argument("--no-fp32", action="store_true", help="rates workload: BF16 only")
    ap.add_argument("--n-streams", type=int, default=128, help="streams (serving workload)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="strain per stream in the throughput phase")
    ap.add_argument("--n-shift", type=int, default=100, help="timeslides per segment (timeslides workload)")
    ap.add_argument("--n-seg", type=int, default=40, help="segments (timeslides workload)")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16"],
                    help="default: fp32 for hour and plain64, bf16 for timeslides")
    ap.add_argument("--ref-windows", type=int, default=32)
    ap.add_argument("--n-win", type=int, default=0, help="analyse this many windows instead (smaller workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16 comparison of the FP32 workload")
    ap.add_argument("--no-tune", action="store_true", help="keep the default conv tiles (no autotuning)")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: skip the nested timeslide-batch (BF16 batched) measurement")
    ap.add_argument("--no-serving", action="store_true",
                    help="default workload: skip the nested serving (p50/p99 latency) measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.precision is None:
        args.precision = "bf16" if args.workload == "timeslides" else "fp32"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "timeslides":
        return run_timeslides(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "resample":
        return run_resample(args)
    if args.workload == "rates":
        return run_rates(args)
    if args.workload == "whiten":
        return run_whiten(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
