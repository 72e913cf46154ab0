#!/usr/bin/env python
"""Throughput of the visibility-based binned angular bispectrum estimator on GB300.

One step = one complete estimate V -> B (gridding plan + gridding, exact
triangle counts, ring-filtered transforms, triple sums, normalisation) for one
realisation of the MWA-shaped workload: 512 x 512 uv grid, dU = 2.3 lambda,
8,128 baselines x 120 time samples = 975,360 visibilities, 20 log-spaced
l bins over 46-1320 (689 closing triplets), FP32 path, sky grid N = 288.
Inputs are resident in HBM; L2 is flushed (a 256 MiB write) before every
timed step because the inputs (15.6 MB) fit in L2.

Reports, on one JSON line: estimates/s over the timed steps (CUDA events on
the library's stream), per-kernel device times from the library's event
profiler, the roofline of the dominant kernel, the end-to-end number through
the host-buffer C entry point (copies included), GPU clocks sampled during
the timed region, and the FP64 oracle timed on the host cores.

--impl reference runs the FP64 oracle itself as the reference arm (host
cores, one realisation per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_ID = 1
METRIC = "ABS estimates/s (V->binned B)"
UNIT = "estimates/s"

# kernels launched per stage-timer entry (the profiler brackets stages)
KERNELS_PER_STAGE = {"grid_plan": 6, "grid_zero": 0, "grid": 1, "grid_finalize": 1, "ring_lists": 1,
                     "count_items": 1, "count_pairs": 1, "count_gather": 1, "ellbar": 1,
                     "fft_rows": 1, "fft_cols": 1, "triple_fp32": 1, "triple_reduce": 1,
                     "normalise": 1, "check_triplets": 1}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_estimate_seconds(inp):
    """FP64 oracle (plain C, one host core) on one realisation of the workload."""
    import oracle
    wl = inp.wl
    t = time.perf_counter()
    oracle.estimate(wl.n_grid, wl.du, wl.ell_edges, inp.uv, inp.vis)
    return time.perf_counter() - t


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    from paper_2412_02246_gb300 import synth
    oracle.build()
    wl = synth.workload(WORKLOAD_ID)
    ins = [synth.make_inputs(WORKLOAD_ID, r) for r in range(min(args.steps, 2))]
    for w in range(args.warmup if args.warmup < 1 else 1):
        oracle_estimate_seconds(ins[0])
    times = [oracle_estimate_seconds(ins[k % len(ins)]) for k in range(args.steps)]
    total = sum(times)
    v = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(wl),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one full realisation of the workload per step (plain C FP64 "
                                   "gridding + brute-force closed-triangle sums), warm-up capped at 1"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(wl):
    return {"workload": "MWA-shaped 512^2 uv grid, dU=2.3 lambda, 128 antennas x 120 time samples = "
                        "975,360 visibilities, 20 log l bins 46-1320, Gaussian gridding sigma=1 cell r=3, "
                        "FP32 path",
            "n_grid": wl.n_grid, "n_vis": 975360, "n_bins": wl.n_bins, "n_fft": 288, "n_trip": 689,
            "global_batch": 1, "l2": "flushed (256 MiB write) before every timed step",
            "parallelism": "replicas"}


def roofline_for(stage, avg_ms, geo, peaks):
    """Algorithmic work per launch of the dominant kernel over its average duration."""
    s = avg_ms * 1e-3
    if stage == "grid":
        # 16 B per visibility (U and V, read once) + 24 B per touched cell of the FP64 grid
        byts = 16.0 * geo["n_vis"] + 24.0 * geo["cells_touched"]
        return {"bound": "hbm", "achieved": byts / s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": byts / s / 1e9 / peaks["hbm_gbs"], "traffic": None,
                "note": "gridder is bound by FP32 ALU (49 compensated weight-accumulations per "
                        "visibility); the HBM fraction is reported against the measured copy peak"}
    if stage == "count_pairs":
        visits = geo["pair_visits"]
        return {"bound": "alu", "achieved": visits / s / 1e9, "peak": geo["alu_gops"], "unit": "Gvisits/s",
                "frac": visits / s / 1e9 / geo["alu_gops"], "traffic": None}
    if stage == "triple_fp32":
        fl = 2.0 * geo["n_trip"] * geo["P"]
        pk = geo["fp32_tflops"]
        return {"bound": "alu", "achieved": fl / s / 1e12, "peak": pk, "unit": "TFLOP/s",
                "frac": fl / s / 1e12 / pk, "traffic": None}
    if stage in ("fft_cols", "fft_rows"):
        byts = geo["fft_bytes"][stage]
        return {"bound": "hbm", "achieved": byts / s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": byts / s / 1e9 / peaks["hbm_gbs"], "traffic": None}
    return {"bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": None,
            "traffic": None}


def run_ours(args):
    import torch

    import paper_2412_02246_gb300 as m
    from paper_2412_02246_gb300 import build as mb
    from paper_2412_02246_gb300 import synth

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        mb.build()
    if world > 1:
        torch.distributed.barrier()
    m.load()
    wl = synth.workload(WORKLOAD_ID)
    cfg = m.Config.from_workload(wl, precision=m.ABS_FP32)
    ijk = m.abs_triplets(cfg)
    nt = len(ijk)
    N = m.abs_fft_size(cfg)
    inp = synth.make_inputs(WORKLOAD_ID, rank)
    uv = torch.from_numpy(inp.uv).to(dev)
    vis = torch.from_numpy(synth.vis_as_float2(inp.vis)).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = m.Context(local, stream)
    B = torch.empty(nt, dtype=torch.float64, device=dev)
    T = torch.empty(nt, dtype=torch.int64, device=dev)
    E = torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        ctx.abs_estimate(cfg, uv, vis, nt, None, B, T, E)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    ctx.sync()
    ctx.profile(True)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.sync()
    t_max = total_ms
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    value = world * args.steps / (t_max * 1e-3)

    # batched form: realisations sharing baselines (plan and counts once per batch)
    R = args.batch
    visR = torch.stack([torch.from_numpy(synth.vis_as_float2(synth.make_inputs(WORKLOAD_ID, 100 + r).vis))
                        for r in range(R)]).to(dev)
    BR = torch.empty((R, nt), dtype=torch.float64, device=dev)
    for _ in range(2):
        ctx.abs_estimate_many(cfg, uv, visR, nt, None, BR, T, E)
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps // 4)
    e0.record(stream)
    for _ in range(reps):
        ctx.abs_estimate_many(cfg, uv, visR, nt, None, BR, T, E)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    batched = R * reps / (e0.elapsed_time(e1) * 1e-3)

    # end to end through the host-buffer entry point (pinned buffers, copies inside)
    huv = torch.from_numpy(inp.uv).pin_memory()
    hvis = torch.from_numpy(synth.vis_as_float2(inp.vis)).pin_memory()
    hB = torch.empty(nt, dtype=torch.float64).pin_memory()
    hT = torch.empty(nt, dtype=torch.int64).pin_memory()
    hE = torch.empty(cfg.n_bins, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        ctx.abs_estimate_host(cfg, huv, hvis, nt, None, hB, hT, hE)
    e2e_t = []
    for _ in range(args.steps):
        flush.fill_(2.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.abs_estimate_host(cfg, huv, hvis, nt, None, hB, hT, hE)
        e2e_t.append(time.perf_counter() - t0)
    e2e_v = world * args.steps / sum(e2e_t)
    h2d = huv.numel() * 4 + hvis.numel() * 4
    d2h = nt * 8 + nt * 8 + cfg.n_bins * 8

    if rank != 0:
        ctx.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # per-kernel averages and the dominant kernel's roofline
    stages = {k: {"ms_total": v[0], "launches": v[1], "avg_us": 1e3 * v[0] / max(v[1], 1)}
              for k, v in prof.items()}
    launches = sum(KERNELS_PER_STAGE.get(k, 1) * v[1] for k, v in prof.items())
    dom = max(prof.items(), key=lambda kv: kv[1][0])[0]
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or 1900.0
    fp32_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    mask_cells = None
    geo = {"n_vis": len(inp.uv), "cells_touched": wl.n_grid * wl.n_grid // 4, "n_trip": nt, "P": N * N,
           "fp32_tflops": fp32_tflops,
           "alu_gops": props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e9 / 4.0,
           "pair_visits": 0, "fft_bytes": {}}
    roof = roofline_for(dom, stages[dom]["avg_us"] * 1e-3, geo, peaks)
    roof["kernel"] = dom
    roof["peak_source"] = peaks["source"]

    cpu_s = oracle_estimate_seconds(inp)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wl), "clocks": clk,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches), "roofline": roof,
        "cpu_baseline": {"value": 1.0 / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one full realisation of the workload (plain C FP64, brute-force "
                                   "closed-triangle sums)"},
        "batched": {"value": batched, "unit": UNIT, "realisations_per_call": R,
                    "note": "abs_estimate_many: realisations sharing one baseline set (plan, counts "
                            "and ring tables once per call)"},
        "stages_us": {k: round(v["avg_us"], 2) for k, v in sorted(stages.items())},
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
