#!/usr/bin/env python
"""Throughput of the visibility-based binned angular bispectrum estimator on GB300.

One step = one complete estimate V -> B (gridding plan + gridding, exact
triangle counts, ring-filtered transforms, split-BF16 triple sums on the
tensor cores, normalisation) for EVERY channel of the multi-channel
workload: 32 channels evenly over 139-169 MHz, each a 4096 x 4096 uv grid
with dU = 0.6 lambda and 10^7 visibilities (one baseline set scaled by
nu / 154.25 MHz), 128 log-spaced l bins over 46-1320 (109,157 closing
triplets), sky grid N = 1080, run as one abs_estimate_batched call (one
CUDA graph over four lanes).  The 5.1 GB of inputs are resident in HBM and
larger than L2, so no flush is needed between steps.

Reports, on one JSON line: estimates/s (channels/s) over the timed steps
(CUDA events on the library's stream); the plain FP32 form on the same
channels and GPU; the end-to-end rate through abs_estimate_batched_host
(host buffers, copies inside); per-kernel device times from one eager
pass with the library's event profiler; the dominant kernel's roofline
from algorithmic bytes / flops; GPU clocks sampled during the timed region;
and the FP64 oracle timed on the host cores on a bounded, stated sample.
Smaller workloads (the MWA-shaped 512^2 estimate, realisation batches, the
uneven 256-item batch, the visibility simulator) are reported beside it.

--impl reference runs the FP64 oracle itself as the reference arm (host
cores, a bounded sample of one channel's estimate per step, scaled).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mproc
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_ID = 4
METRIC = "ABS estimates/s (V→binned B) & triplet TFLOP/s, vs plain FP32 at ≤3e-4 rel err"
UNIT = "estimates/s"

# kernels launched per stage-timer entry (the profiler brackets stages); the
# gridding plan runs the key kernel and, per radix pass of up to 11-bit digits
# of the (uv tile, cell) key, a scan and a scatter (which counts the next
# pass's histogram); the ring lists run cells and finish; the pair counts run
# once per byte map (filled, annulus)
KERNELS_PER_STAGE = {"grid_zero": 0, "grid": 1, "grid_finalize": 1, "grid_mask": 1, "ring_lists": 2,
                     "count_items": 1, "count_pairs": 2, "count_gather": 1, "ellbar": 2,
                     "fft_rows": 1, "fft_cols": 1, "triple_fp32": 1, "triple_reduce": 1,
                     "normalise": 1, "check_triplets": 1, "tc_split": 1, "tc_pad": 1, "triple_tc": 1,
                     "tc_reduce": 2}


def plan_kernels(n_grid, radius):
    tiles = -(-(n_grid - 1 + 2 * radius) // 16)
    passes = -(-int(tiles * tiles * 256).bit_length() // 11)   # keys: (tile, cell in the tile)
    return 1 + 2 * passes


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", 1700.0),
                "sm_max_mhz": d.get("sm_max_mhz"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": None,
            "source": "fallback"}


# DRAM traffic of one launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures of the kernel on the named workload, with the SHA-256 of the source
# file the kernel was built from when it was captured.  A kernel whose source has
# changed since then reports null.
MEASURED_TRAFFIC = {
    "fft_rows": {"bytes": 1250012000, "source": "paper_2412_02246_gb300/csrc/fft.cu",
                 "sha256": "e0c763502d9680073163ddc3c914101553e28b3b6d52983992aa0a07de5173b0"},
    "triple_tc": {"bytes": 1339430000, "source": "paper_2412_02246_gb300/csrc/triple_tc.cu",
                  "sha256": "56ec114d7a18bc151efae201334e7ece346d772bb2221b660021b47bf0ef0815"},
}


def measured_traffic(stage):
    e = MEASURED_TRAFFIC.get(stage)
    if e is None:
        return None
    import hashlib
    path = os.path.join(ROOT, e["source"])
    if not os.path.exists(path) or hashlib.sha256(open(path, "rb").read()).hexdigest() != e["sha256"]:
        return None
    return e["bytes"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while active."""

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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def whole_job_rate(total_ms, steps, world, dev, units_per_step=1):
    """Whole-job units/s over all ranks: every rank ran `steps` steps of
    `units_per_step` independent estimates in `total_ms`; the job takes as long
    as its slowest rank (MAX over ranks), and the units are those of all ranks.
    Returns (rate, max_ms)."""
    import torch
    t_max = float(total_ms)
    if world > 1:
        t = torch.tensor([t_max], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    return world * steps * units_per_step / (t_max * 1e-3), t_max


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def make_pool(workers):
    """A spawn-context process pool (made before this process's first CUDA call)."""
    return mproc.get_context("spawn").Pool(workers)


# ----------------------------------------------------------------------------- inputs


def _channel_job(args):
    """One channel's seeded inputs, as (channel, uv float32 [n, 2], vis float32 [n, 2])."""
    ch, realisation = args
    from paper_2412_02246_gb300 import synth
    inp = synth.channel_inputs(ch, realisation=realisation, wl=synth.workload(WORKLOAD_ID))
    return ch, inp.uv, synth.vis_as_float2(inp.vis)


def _batch_job(i):
    """Item i of the seeded 256-item uneven batch, as (i, workload, uv, vis)."""
    from paper_2412_02246_gb300 import synth
    rng = np.random.default_rng(2412)
    for k in range(i + 1):
        w = synth.batch_item(rng, k)
    inp = synth.make_inputs(3, i, wl=w)
    return i, w, inp.uv, synth.vis_as_float2(inp.vis)


# ----------------------------------------------------------------------------- oracle timing


def _grid_part(args):
    """Oracle gridding of one slice in a spawned worker: (seconds for no visibilities, seconds
    for the slice, slice length); the grids stay in the worker (only times come back)."""
    n, du, uv, vis = args
    import oracle
    oracle.grid(8, du, uv[:1], vis[:1])      # loads the library before anything is timed
    t0 = time.perf_counter()
    oracle.grid(n, du, uv[:0], vis[:0])
    t1 = time.perf_counter()
    oracle.grid(n, du, uv, vis)
    t2 = time.perf_counter()
    oracle.grid(n, du, uv[:0], vis[:0])
    t3 = time.perf_counter()
    return min(t1 - t0, t3 - t2), t2 - t1, len(uv)


def oracle_grid_sample(uv, vis2, wl, pool, cores, m):
    """Seconds the FP64 oracle's gridding (plain C) takes for all of a channel's
    visibilities on `cores` processes, from the first m of them split over `cores`
    spawned workers: each worker's per-visibility time (its slice minus an empty call,
    which is the grid's fixed cost) times the visibilities a worker would take, plus the
    fixed cost, plus the time to add the workers' grids (measured on the parent's grid).
    Returns (seconds, the Grid of the m visibilities made in this process, untimed)."""
    import oracle
    m = min(m, len(uv))
    vis = (vis2[:m, 0].astype(np.float64) + 1j * vis2[:m, 1].astype(np.float64)).astype(np.complex64)
    parts = [p for p in np.array_split(np.arange(m), cores) if len(p)]
    res = pool.map(_grid_part, [(wl.n_grid, wl.du, uv[p], vis[p]) for p in parts])
    fixed = max(r[0] for r in res)
    per_vis = float(np.mean([(r[1] - r[0]) / r[2] for r in res]))
    gr = oracle.grid(wl.n_grid, wl.du, uv[:m], vis)
    t0 = time.perf_counter()
    acc = gr.grid.copy()
    for _ in range(len(parts) - 1):
        acc += gr.grid
    t_add = (time.perf_counter() - t0) * 2      # complex sums plus the weight and count planes
    return fixed + per_vis * len(uv) / len(parts) + t_add, gr


def j_products(ijk):
    """Per middle ring j: rows x columns of the matrix product the oracle's FFT form takes for it."""
    out = {}
    for j in np.unique(ijk[:, 1]):
        s = ijk[ijk[:, 1] == j]
        out[int(j)] = (int(s[:, 0].max()) - int(s[:, 0].min()) + 1) * (int(s[:, 2].max()) - int(s[:, 2].min()) + 1)
    return out


class OracleSampler:
    """Seconds the FP64 oracle takes for one channel's whole estimate, from timed samples:
    gridding of a slice of the visibilities over all host cores (scaled to every
    visibility), the FFT-form fields of every ring, data and unit mask (timed once, in
    full, from the gridded slice: a transform costs the same whatever the values), and
    the FFT-form sums and counts of a few middle rings (scaled by their share of the
    matrix-product work)."""

    def __init__(self, uv, vis2, wl, pool, cores, m):
        import oracle
        self.uv, self.vis2, self.wl, self.pool, self.cores, self.m = uv, vis2, wl, pool, cores, m
        self.t_grid, gr = oracle_grid_sample(uv, vis2, wl, pool, cores, m)
        X, f = oracle.mean_grid(gr)
        self.q = oracle.ring_q(wl.ell_edges, wl.du)
        self.ijk = oracle.triplets(self.q)
        self.N = oracle.min_fft_size(self.q, wl.n_grid)
        t0 = time.perf_counter()
        D, _ = oracle.ring_fields(X, f, self.q, self.N)
        I, _ = oracle.ring_fields(X, f, self.q, self.N, unit=True)
        self.t_fields = time.perf_counter() - t0
        self.fields = (D, I)
        self.jp = j_products(self.ijk)

    def seconds(self, js, regrid=False):
        import oracle
        if regrid:
            self.t_grid, _ = oracle_grid_sample(self.uv, self.vis2, self.wl, self.pool, self.cores, self.m)
        t_grid = self.t_grid
        js = [j for j in js if j in self.jp]
        sel = np.isin(self.ijk[:, 1], js)
        t0 = time.perf_counter()
        oracle.fft_form_all(None, None, None, self.ijk[sel], self.N, fields=self.fields)
        t_sums = (time.perf_counter() - t0) * sum(self.jp.values()) / max(1, sum(self.jp[j] for j in js))
        return t_grid + self.t_fields + t_sums, {"grid_s": round(t_grid, 3), "fields_s": round(self.t_fields, 3),
                                                 "sums_s": round(t_sums, 3)}


def workload_config(n_chan):
    return {"workload": f"multi-channel: {n_chan} channels 139-169 MHz, 4096^2 uv grid, dU=0.6 lambda, 1e7 "
                        "visibilities per channel (one baseline set scaled by nu/154.25 MHz), diffuse + 2,000 "
                        "point-source sky, 128 log l bins 46-1320 (109,157 triplets), sky grid N=1080, Gaussian "
                        "gridding sigma=1 cell r=3, split-BF16 triple sums, FP64 counts and normalisation",
            "n_grid": 4096, "n_vis_per_channel": 10_000_000, "channels_per_step": n_chan, "n_bins": 128,
            "n_fft": 1080, "n_trip": 109157, "global_batch": n_chan,
            "l2": "inputs larger than L2 (5.1 GB resident per 32-channel step), no flush",
            "parallelism": "replicas (each rank estimates its own realisation of every channel)"}


# ----------------------------------------------------------------------------- roofline


def ring_census(mask, q, n):
    """Lattice cells (A) and filled cells (F) of every ring on an n x n FFT-ordered grid."""
    k = np.arange(n, dtype=np.int64)
    k = np.where(k > n // 2, k - n, k)
    on = np.abs(k) <= n // 2 - 1
    r2 = k[None, :] ** 2 + k[:, None] ** 2
    inr = (r2 >= q[0]) & (r2 < q[-1]) & on[None, :] & on[:, None]
    ring = np.searchsorted(np.asarray(q), r2[inr], side="right") - 1
    nb = len(q) - 1
    A = np.bincount(ring, minlength=nb)
    F = np.bincount(ring[mask[inr] > 0], minlength=nb)
    return A.astype(np.int64), F.astype(np.int64)


def count_route_visits(A, F):
    """Pair visits of the exact count kernel, which takes the cheaper of its two routes: the
    direct enumeration of the filled cells, sum over a <= b of floor(F_a / 2) F_b, or the
    holes route (H = A - F), sum over a <= b of floor(H_a / 2) A_b + 2 floor(F_a / 2) H_b
    (the full-annulus table it subtracts from is computed once per configuration)."""
    H = A - F
    tail = lambda v: np.cumsum(v[::-1])[::-1]          # sum over b >= a
    direct = int(np.sum((F // 2) * tail(F)))
    holes = int(np.sum((H // 2) * tail(A) + 2 * (F // 2) * tail(H)))
    return holes if holes < direct else direct


def ring_rmax(q, half):
    """Per ring, the largest |g_x| of a lattice cell on the grid (-1: no cell), as the library derives it."""
    import math
    out = []
    for a in range(len(q) - 1):
        lo, hi, r = int(q[a]), int(q[a + 1]) - 1, -1
        if hi >= lo:
            for x in range(min(half, math.isqrt(hi)), -1, -1):
                ylo = math.isqrt(lo - x * x - 1) + 1 if lo - x * x > 0 else 0
                yhi = min(half, math.isqrt(hi - x * x))
                if ylo <= yhi:
                    r = x
                    break
        out.append(r)
    return out


def pair_lines(q, n):
    """Columns of the first transform pass: 2 R_p + 1 per ring pair p (R_p its largest |g_x|)."""
    rm = ring_rmax(q, n // 2 - 1)
    nb = len(q) - 1
    return sum(2 * r + 1 for r in (max(rm[a], rm[a + 1] if a + 1 < nb else -1) for a in range(0, nb, 2)) if r >= 0)


def algorithmic_work(stage, geo):
    """Algorithmic work of one launch of `stage` for one estimate, in its roofline's unit.

    grid:        HBM bytes, 16 per visibility read (8 B position + 8 B value) and 13 per uv
                 cell written (8 B complex value + 4 B weight + 1 B filled state)
    fft_cols:    HBM bytes, 24 per filled ring cell read (FP64 re, im, weight sums) and 8 per
                 transformed point written ((2 R_p + 1) N points per ring pair, FP32 complex
                 on the split-BF16 path, 16 B double-float on the FP32 path)
    fft_rows:    HBM bytes, those points read back and, per field value, 4 written (FP32
                 fields) or 8 (the split-BF16 planes the estimate's row pass writes: BF16 hi
                 and lo, FP32 copy)
    triple_tc:   BF16 tensor flops, 3 products x 2 flops per (closing triplet, pixel)
    triple_fp32: FP32 flops, 2 per (closing triplet, pixel)
    count_pairs: integer lane-ops, 2 per pair visit of the route the kernel takes
    """
    P, nt, pt = geo["P"], geo["n_trip"], geo.get("point_bytes", 8)
    if stage == "grid":
        return "hbm", 16.0 * geo["n_vis"] + 13.0 * geo["cells"]
    if stage == "fft_cols":
        return "hbm", 24.0 * geo["filled"] + pt * geo["lines"] * geo["N"]
    if stage == "fft_rows":
        return "hbm", pt * geo["lines"] * geo["N"] + geo.get("field_bytes", 4) * geo["nb"] * P
    if stage == "triple_tc":
        return "tensor", 6.0 * nt * P
    if stage == "triple_fp32":
        return "fp32", 2.0 * nt * P
    if stage == "count_pairs":
        return "alu", 2.0 * geo["pair_visits"]
    return None, None


def roofline(stage, avg_ms, geo, peaks, clk_mhz, sms):
    """Roofline of one kernel: achieved = algorithmic work of one launch / its average duration."""
    kind, work = algorithmic_work(stage, geo)
    if kind is None:
        return None
    s = avg_ms * 1e-3
    if kind == "hbm":
        out = {"bound": "hbm", "achieved": work / s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "peak_source": peaks["source"] + " (HBM copy)"}
    elif kind == "tensor":
        out = {"bound": "tensor", "achieved": work / s / 1e12, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
               "peak_source": peaks["source"] + " (cuBLAS bf16, burst)"}
    else:
        if not clk_mhz:
            return {"bound": "alu", "achieved": None, "peak": None, "frac": None,
                    "unit": "TFLOP/s" if kind == "fp32" else "Tlane-op/s", "note": "no SM clock sample"}
        lanes = sms * 128 * clk_mhz * 1e6
        peak = 2 * lanes if kind == "fp32" else lanes
        out = {"bound": "alu", "achieved": work / s / 1e12, "peak": peak / 1e12,
               "unit": "TFLOP/s" if kind == "fp32" else "Tlane-op/s",
               "peak_source": f"derived: {sms} SMs x 128 lanes x {clk_mhz:.0f} MHz median sampled SM clock"
                              + (" x 2 flops per FMA" if kind == "fp32" else "")}
    out["frac"] = out["achieved"] / out["peak"]
    out["work_per_launch"] = work
    return out


def channel_geometry(m, cfg, ctx, items, torch, dev):
    """Per-channel averages of what the rooflines need: filled ring cells and pair visits."""
    n = cfg.n_grid
    q = m.abs_ring_q(cfg)
    mk = torch.empty((n, n), dtype=torch.uint8, device=dev)
    g = torch.empty((n, n, 2), dtype=torch.float32, device=dev)
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    visits = fills = 0
    for it in items:
        ctx.abs_grid(cfg, it[1], it[2], g, w, mk)
        ctx.sync()
        A, F = ring_census(mk.cpu().numpy(), q, n)
        visits += count_route_visits(A, F)
        fills += int(F.sum())
    N = m.abs_fft_size(cfg)
    k = len(items)
    return {"pair_visits": visits / k, "filled": fills / k, "n_trip": len(m.abs_triplets(cfg)), "P": N * N,
            "N": N, "nb": cfg.n_bins, "n_vis": int(items[0][1].shape[0]), "cells": n * n,
            "lines": pair_lines(q, n), "point_bytes": 8 if cfg.precision == m.ABS_SPLIT_BF16 else 16,
            "field_bytes": 8 if cfg.precision == m.ABS_SPLIT_BF16 else 4}


# ----------------------------------------------------------------------------- reference arm


REF_SAMPLE = ("per step, one channel of the multi-channel workload: oracle gridding (plain C, FP64) of a "
              "{m}-visibility slice split over the host cores (per-visibility time scaled to 1e7 visibilities, "
              "plus the grid's fixed cost and the sum of the per-core grids); FFT-form fields "
              "(FP64 FFT on all cores) of all 128 rings, data and unit mask, timed once in full; FFT-form sums "
              "and counts (FP64 matrix products, multi-threaded BLAS) of {j} middle rings, scaled by their "
              "share of the products")


def run_reference(args):
    """The FP64 oracle as the reference arm: per step a bounded sample of one channel's
    estimate on the host cores, scaled to the whole estimate; value = estimates/s."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = cpu_cores()
    pool = make_pool(cores)
    _, uv, vis2 = _channel_job((0, 0))
    from paper_2412_02246_gb300 import synth
    wl = synth.workload(WORKLOAD_ID)
    smp = OracleSampler(uv, vis2, wl, pool, cores, 1_000_000)
    js = sorted(smp.jp, key=lambda j: -smp.jp[j])[:len(smp.jp) // 2]   # the heavier half of the middle rings
    times, parts = [], None
    for k in range(max(args.warmup, 0) + args.steps):
        t, parts = smp.seconds([js[(17 * k) % len(js)], js[(17 * k + 7) % len(js)]], regrid=True)
        if k >= max(args.warmup, 0):
            times.append(t)
    pool.close()
    total = sum(times)
    v = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(workload_config(1), global_batch=1),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": REF_SAMPLE.format(m="1,000,000", j=2), "parts_s_last_step": parts},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm


def timed_calls(fn, steps, stream, torch, dev, before=None):
    """Device milliseconds of `steps` calls of fn, each bracketed by CUDA events on `stream`
    (before(), if given, runs ahead of each start event: an L2 flush)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        if before:
            before()
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    return [a.elapsed_time(b) for a, b in ev]


def max_rel_big(B, Bref):
    """Max relative difference over triplets with |Bref| >= 1e-3 max |Bref| (and equal NaN pattern)."""
    ok = ~np.isnan(Bref)
    if not ok.any():
        return 0.0
    big = ok & (np.abs(Bref) >= 1e-3 * np.max(np.abs(Bref[ok])))
    return float(np.max(np.abs(B[big] - Bref[big]) / np.abs(Bref[big])))


def mwa_extras(m, synth, ctx, torch, dev, stream, steps, rank):
    """The MWA-shaped 512^2 workload (975,360 visibilities, 20 rings, 689 triplets, N = 288):
    one estimate per call, FP32 and split-BF16 (graph replays, L2 flushed before each), end
    to end through abs_estimate_host, and 16 realisations per abs_estimate_many call."""
    wl = synth.workload(1)
    inp = synth.make_inputs(1, rank)
    uv = torch.from_numpy(inp.uv).to(dev)
    vis = torch.from_numpy(synth.vis_as_float2(inp.vis)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": "MWA-shaped 512^2 uv grid, dU=2.3 lambda, 128 antennas x 120 samples = 975,360 "
                       "visibilities, 20 log l bins, 689 triplets, N=288 (L2 flushed before every call)"}
    for name, prec in (("fp32", m.ABS_FP32), ("split_bf16", m.ABS_SPLIT_BF16)):
        cfg = m.Config.from_workload(wl, precision=prec)
        nt = len(m.abs_triplets(cfg))
        B = torch.empty(nt, dtype=torch.float64, device=dev)
        T = torch.empty(nt, dtype=torch.int64, device=dev)
        E = torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)
        for _ in range(3):
            ctx.abs_estimate(cfg, uv, vis, nt, None, B, T, E)
        ctx.sync()

        t = timed_calls(lambda: ctx.abs_estimate(cfg, uv, vis, nt, None, B, T, E), steps, stream, torch, dev,
                        before=lambda: flush.fill_(1.0))
        out[name] = {"value": steps / (sum(t) * 1e-3), "unit": UNIT}
        if prec == m.ABS_FP32:
            huv, hvis = torch.from_numpy(inp.uv).pin_memory(), torch.from_numpy(synth.vis_as_float2(inp.vis)).pin_memory()
            hB = torch.empty(nt, dtype=torch.float64).pin_memory()
            hT = torch.empty(nt, dtype=torch.int64).pin_memory()
            hE = torch.empty(cfg.n_bins, dtype=torch.float64).pin_memory()
            for _ in range(3):
                ctx.abs_estimate_host(cfg, huv, hvis, nt, None, hB, hT, hE)
            e2e = []
            for _ in range(steps):
                flush.fill_(2.0)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                ctx.abs_estimate_host(cfg, huv, hvis, nt, None, hB, hT, hE)
                e2e.append(time.perf_counter() - t0)
            out[name]["e2e"] = steps / sum(e2e)
            R = 16
            visR = torch.stack([torch.from_numpy(synth.vis_as_float2(synth.make_inputs(1, 100 + r).vis))
                                for r in range(R)]).to(dev)
            BR = torch.empty((R, nt), dtype=torch.float64, device=dev)
            for _ in range(3):
                ctx.abs_estimate_many(cfg, uv, visR, nt, None, BR, T, E)
            ctx.sync()
            tb = timed_calls(lambda: ctx.abs_estimate_many(cfg, uv, visR, nt, None, BR, T, E), max(2, steps // 4),
                             stream, torch, dev)
            out["realisations_16"] = {"value": R * len(tb) / (sum(tb) * 1e-3), "unit": UNIT,
                                      "note": "abs_estimate_many: 16 realisations sharing one baseline set"}
            cells = [torch.empty((cfg.n_bins, 5, 5), dtype=torch.float64, device=dev) for _ in range(3)]
            ctx.abs_rebin(cfg, BR, T, E, None, 5, 5, *cells)
            tr = timed_calls(lambda: ctx.abs_rebin(cfg, BR, T, E, None, 5, 5, *cells), 5, stream, torch, dev)
            out["rebin_us_16x689"] = round(1e3 * sum(tr) / len(tr), 2)
    return out


def uneven_extras(m, ctx, batch_inputs, torch, dev, stream, steps):
    """Every item of the seeded 256-item uneven batch in one abs_estimate_batched call."""
    items = []
    for i, w, uv, vis in batch_inputs:
        cfg = m.Config.from_workload(w)
        nt = len(m.abs_triplets(cfg))
        items.append((cfg, torch.from_numpy(uv).to(dev), torch.from_numpy(vis).to(dev), nt, None,
                      torch.empty(nt, dtype=torch.float64, device=dev),
                      torch.empty(nt, dtype=torch.int64, device=dev),
                      torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)))
    for _ in range(3):   # eager (autotuning, workspaces), capture, replay
        ctx.abs_estimate_batched(items)
    ctx.sync()
    t = timed_calls(lambda: ctx.abs_estimate_batched(items), max(2, steps // 2), stream, torch, dev)

    # the same items one after another on the context's stream, each replayed from its own graph
    def serial():
        for it in items:
            ctx.abs_estimate(*it)
    for _ in range(3):
        serial()
    ctx.sync()
    ts = timed_calls(serial, max(2, steps // 2), stream, torch, dev)
    return {"value": len(items) * len(t) / (sum(t) * 1e-3), "unit": UNIT, "items_per_call": len(items),
            "ms_per_call": sum(t) / len(t),
            "serial": {"value": len(items) * len(ts) / (sum(ts) * 1e-3), "unit": UNIT, "ms": sum(ts) / len(ts),
                       "note": "the same items through abs_estimate one after another on one stream"},
            "note": "abs_estimate_batched over the seeded uneven batch: grids {256,512,1024}^2, 1e5-1e6 "
                    "visibilities, 16-48 log l bins, split-BF16, one CUDA graph over four lanes"}


def simulator_extras(m, synth, ctx, uv, torch, dev, stream):
    msim, nsim = 256, 100_000
    sky = torch.from_numpy(synth.quadratic_sky(synth.gaussian_field(msim, np.random.default_rng(5)), 0.3)
                           .astype(np.float32)).to(dev)
    vsim = torch.empty((nsim, 2), dtype=torch.float32, device=dev)
    dth = float(np.deg2rad(0.029))
    d_over_lam = 4.0 / (299792458.0 / 154.25e6)
    ctx.abs_simulate_vis(sky, dth, uv[:nsim], vsim, m.ABS_BEAM_MWA_TILE, d_over_lam)
    t = timed_calls(lambda: ctx.abs_simulate_vis(sky, dth, uv[:nsim], vsim, m.ABS_BEAM_MWA_TILE, d_over_lam), 1,
                    stream, torch, dev)
    s = t[0] * 1e-3
    return {"vis_per_s": nsim / s, "phase_terms_per_s": nsim * msim * msim / s, "ms": s * 1e3, "n_vis": nsim,
            "map": msim, "note": "abs_simulate_vis: MWA tile beam, 0.029 deg pixels, direct DFT"}


def cube_extras(m, synth, ctx, torch, dev, stream, steps, peaks):
    """The multi-frequency (3-D) form on the MWA-shaped cube: 32 channels of 975,360 visibilities
    (139-169 MHz), 512^2 grid, 20 log l rings x 4 |delay| bins, 18,603 bin triplets, N = 288,
    N_z = 46; one abs_estimate_3d per call (graph replays; the 500 MB of inputs exceed L2),
    FP32 and split-BF16, and one eager call of each with the stage profiler."""
    ci = synth.cube_inputs(6)
    uv = torch.from_numpy(np.ascontiguousarray(ci.uv)).to(dev)
    vis = torch.from_numpy(np.ascontiguousarray(ci.vis).view(np.float32).reshape(ci.vis.shape + (2,))).to(dev)
    out = {"workload": "MWA-shaped cube: 32 channels x 975,360 visibilities (139-169 MHz, baselines scaled by "
                       "nu / 154.25 MHz), 512^2 uv grid, dU=2.3 lambda, 20 log l rings x |delay| bins {0}, [1,4), "
                       "[4,8), [8,16): 80 bins, 18,603 bin triplets, N=288, N_z=46 (3.82e6 voxels)"}
    res = {}
    for name, prec in (("fp32", m.ABS_FP32), ("split_bf16", m.ABS_SPLIT_BF16)):
        cfg = m.Config3D.from_cube(ci, precision=prec)
        nt = len(m.abs_triplets_3d(cfg))
        B = torch.empty(nt, dtype=torch.float64, device=dev)
        T = torch.empty(nt, dtype=torch.int64, device=dev)
        E = torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)
        for _ in range(3):
            ctx.abs_estimate_3d(cfg, uv, vis, nt, None, B, T, E)
        ctx.sync()
        t = timed_calls(lambda: ctx.abs_estimate_3d(cfg, uv, vis, nt, None, B, T, E), steps, stream, torch, dev)
        res[name] = (B.cpu().numpy(), T.cpu().numpy())
        torch.cuda.nvtx.range_push(f"cube_profile_{name}")
        ctx.profile(True)
        ctx.abs_estimate_3d(cfg, uv, vis, nt, None, B, T, E)
        prof = ctx.profile_read()
        ctx.profile(False)
        torch.cuda.nvtx.range_pop()
        P3 = 288 * 288 * 46
        o = {"value": steps / (sum(t) * 1e-3), "unit": UNIT, "ms": sum(t) / steps,
             "stages_us": {k: round(1e3 * v[0], 1) for k, v in sorted(prof.items())}}
        if "triple_tc" in prof:
            ms = prof["triple_tc"][0]
            useful = 6.0 * nt * P3
            o["triple_tc"] = {"ms": ms, "useful_bf16_tflops": useful / (ms * 1e9),
                              "frac_useful_of_measured_bf16": useful / (ms * 1e9) / peaks["bf16_tflops"]}
        if "triple_fp32" in prof:
            ms = prof["triple_fp32"][0]
            o["triple_fp32"] = {"ms": ms, "fp32_tflops": 2.0 * nt * P3 / (ms * 1e9)}
        out[name] = o
    out["split_vs_fp32_max_rel_err"] = max_rel_big(res["split_bf16"][0], res["fp32"][0])
    out["counts_equal"] = bool(np.array_equal(res["split_bf16"][1], res["fp32"][1]))
    out["split_bf16_over_fp32"] = out["split_bf16"]["value"] / out["fp32"]["value"]
    return out


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    cores = cpu_cores()
    # inputs first, made in spawned workers before this process's first CUDA call
    pool = make_pool(max(1, min(cores, 16)))
    chan_inputs = sorted(pool.map(_channel_job, [(c, rank) for c in range(args.channels)]), key=lambda r: r[0])
    batch_inputs = []
    if rank == 0 and args.batch_items > 0:
        batch_inputs = sorted(pool.map(_batch_job, range(args.batch_items)), key=lambda r: r[0])

    import paper_2412_02246_gb300 as m
    from paper_2412_02246_gb300 import build as mb
    from paper_2412_02246_gb300 import synth

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
    # a stream of our own (the library captures CUDA graphs on it; the legacy
    # default stream cannot be captured)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = m.Context(local, stream)
    wl = synth.workload(WORKLOAD_ID)
    cfg = m.Config.from_workload(wl)
    cfg32 = m.Config.from_workload(wl, precision=m.ABS_FP32)
    assert cfg.precision == m.ABS_SPLIT_BF16
    nt = len(m.abs_triplets(cfg))
    nch = len(chan_inputs)
    uvd = [torch.from_numpy(uv).to(dev) for _, uv, _ in chan_inputs]
    visd = [torch.from_numpy(v).to(dev) for _, _, v in chan_inputs]

    def outputs(c):
        return (torch.empty(nt, dtype=torch.float64, device=dev), torch.empty(nt, dtype=torch.int64, device=dev),
                torch.empty(c.n_bins, dtype=torch.float64, device=dev))
    items = [(cfg, u, v, nt, None) + outputs(cfg) for u, v in zip(uvd, visd)]
    items32 = [(cfg32, u, v, nt, None) + outputs(cfg32) for u, v in zip(uvd, visd)]

    def step():
        ctx.abs_estimate_batched(items)

    for _ in range(args.warmup):   # eager (autotuning, workspaces), capture, replays
        step()
    ctx.sync()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    step_ms = timed_calls(step, args.steps, stream, torch, dev)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    value, t_max = whole_job_rate(sum(step_ms), args.steps, world, dev, nch)

    # the plain FP32 form on the same channels and GPU
    for _ in range(3):
        ctx.abs_estimate_batched(items32)
    ctx.sync()
    s32 = max(2, args.steps // 2)
    t32 = timed_calls(lambda: ctx.abs_estimate_batched(items32), s32, stream, torch, dev)
    fp32_value = nch * s32 / (sum(t32) * 1e-3)
    agree = max(max_rel_big(a[5].cpu().numpy(), b[5].cpu().numpy()) for a, b in zip(items, items32))
    counts_equal = all(torch.equal(a[6], b[6]) for a, b in zip(items, items32))

    # end to end: host buffers (pinned) through abs_estimate_batched_host, copies inside
    h_items = []
    for (_, uv, v) in chan_inputs:
        h_items.append((cfg, torch.from_numpy(uv).pin_memory(), torch.from_numpy(v).pin_memory(), nt, None,
                        torch.empty(nt, dtype=torch.float64).pin_memory(),
                        torch.empty(nt, dtype=torch.int64).pin_memory(),
                        torch.empty(cfg.n_bins, dtype=torch.float64).pin_memory()))
    for _ in range(max(2, args.warmup)):
        ctx.abs_estimate_batched_host(h_items)
    e2e_s = []
    if world > 1:
        torch.distributed.barrier()
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx.abs_estimate_batched_host(h_items)
        e2e_s.append(time.perf_counter() - t0)
    e2e_v, _ = whole_job_rate(1e3 * sum(e2e_s), args.steps, world, dev, nch)
    h2d = sum(it[1].numel() * 4 + it[2].numel() * 4 for it in h_items)
    d2h = nch * (nt * 16 + cfg.n_bins * 8)
    assert torch.equal(h_items[0][6], items[0][6].cpu())
    del h_items

    if rank != 0:
        ctx.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        pool.close()
        return

    # per-kernel device times: one eager pass over every channel with the stage profiler
    # (an NVTX range, so that a profiler can pick these launches)
    torch.cuda.nvtx.range_push("stage_profile")
    ctx.profile(True)
    for it in items:
        ctx.abs_estimate(cfg, it[1], it[2], nt, None, *it[5:])
    torch.cuda.synchronize(dev)
    prof = ctx.profile_read()
    ctx.profile(False)
    torch.cuda.nvtx.range_pop()
    ctx.profile(True)
    for it in items32[:4]:
        ctx.abs_estimate(cfg32, it[1], it[2], nt, None, *it[5:])
    torch.cuda.synchronize(dev)
    prof32 = ctx.profile_read()
    ctx.profile(False)
    ctx.sync()
    per = {k: 1e3 * v[0] / nch for k, v in prof.items()}            # us per channel
    kps = dict(KERNELS_PER_STAGE, grid_plan=plan_kernels(wl.n_grid, wl.radius_cells))
    launches = int(sum(kps.get(k, 1) * v[1] for k, v in prof.items()))
    dom = max((k for k in prof if kps.get(k, 1) == 1), key=lambda k: prof[k][0])
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    geo = channel_geometry(m, cfg, ctx, items, torch, dev)
    avg_ms = lambda k, p=prof: p[k][0] / max(p[k][1], 1)
    roof = roofline(dom, avg_ms(dom), geo, peaks, clk.get("sm_mhz"), sms) or {}
    roof["kernel"] = dom
    roof["traffic"] = measured_traffic(dom)
    others = {}
    for k in ("triple_tc", "count_pairs", "fft_rows", "fft_cols", "grid"):
        if k in prof and k != dom:
            r = roofline(k, avg_ms(k), geo, peaks, clk.get("sm_mhz"), sms)
            if r:
                r["traffic"] = measured_traffic(k)
                others[k] = r
    tc_exec = None
    if "triple_tc" in prof:
        tc_exec = ctx.tuned_shape(cfg)
    geo32 = dict(geo, point_bytes=16, field_bytes=4)
    fp32_triple = roofline("triple_fp32", avg_ms("triple_fp32", prof32), geo32, peaks, clk.get("sm_mhz"), sms) \
        if "triple_fp32" in prof32 else None

    # the FP64 oracle on the host cores, on a bounded sample of channel 0's estimate
    import oracle
    oracle.build()
    _, uv0, v0 = chan_inputs[0]
    smp = OracleSampler(uv0, v0, wl, pool, cores, 2_000_000)
    js = sorted(smp.jp)
    cpu_s, cpu_parts = smp.seconds([js[int(p)] for p in np.linspace(0, len(js) - 1, 12)])
    del smp
    pool.close()

    extras = {}
    extras["mwa512"] = mwa_extras(m, synth, ctx, torch, dev, stream, 20, rank)
    if batch_inputs:
        extras["batched_uneven"] = uneven_extras(m, ctx, batch_inputs, torch, dev, stream, args.steps)
    extras["simulator"] = simulator_extras(m, synth, ctx, uvd[0], torch, dev, stream)
    if rank == 0 and args.cube:
        extras["cube3d"] = cube_extras(m, synth, ctx, torch, dev, stream, max(3, args.steps // 2), peaks)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 (split-BF16 triple sums, FP32 transforms, "
                                                         "FP64 counts and normalisation)",
        "data": "synthetic", "config": workload_config(nch), "clocks": clk,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "entry": "abs_estimate_batched_host (pinned host buffers, copies inside the batch's graph)"},
        "gpu_launches": launches, "roofline": roof, "stage_rooflines": others,
        "cpu_baseline": {"value": 1.0 / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": REF_SAMPLE.format(m="2,000,000", j=12).replace("per step, ", ""),
                         "parts_s": cpu_parts},
        "fp32": {"value": fp32_value, "unit": UNIT, "split_bf16_over_fp32": value / world / fp32_value,
                 "split_vs_fp32_max_rel_err": agree, "counts_equal": counts_equal,
                 "triple_fp32": fp32_triple,
                 "note": "the same channels through the plain FP32 path (SIMT FP32 triple sums with double-float "
                         "partials, double-float transforms) on the same GPU; max relative difference of B over "
                         "triplets with |B| >= 1e-3 max|B|"},
        "triple_tc_shape": tc_exec,
        "stages_us_per_channel": {k: round(v, 1) for k, v in sorted(per.items())},
        "stages_fp32_us_per_channel": {k: round(1e3 * v[0] / 4, 1) for k, v in sorted(prof32.items())},
        "kernel_timing": "stage device times: CUDA events around each stage on the library's stream, one eager "
                         "abs_estimate per channel (graphs off)",
        **extras,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--channels", type=int, default=32, help="channels per step (the workload has 32)")
    ap.add_argument("--batch-items", type=int, default=256, help="items of the uneven batch (0: skip it)")
    ap.add_argument("--cube", type=int, default=1, help="time the multi-frequency (3-D) form too (0: skip it)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
