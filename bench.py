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
the library's stream; the library replays each estimate as a captured CUDA
graph), per-kernel device times from the library's event profiler over the
same number of steps run again eagerly, the roofline of the dominant kernel,
the end-to-end number through the host-buffer C entry point (copies
included), GPU clocks sampled during the timed region, and the FP64 oracle
timed on the host cores.

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

# kernels launched per stage-timer entry (the profiler brackets stages); the
# gridding plan runs the key kernel and, per radix pass of up to 11-bit digits
# of the (uv tile, cell) key, a scan and a scatter (which counts the next
# pass's histogram); the ring lists run cells and finish; the pair counts run
# once per byte map (filled, annulus)
KERNELS_PER_STAGE = {"grid_zero": 0, "grid": 1, "grid_finalize": 1, "grid_mask": 1, "ring_lists": 2,
                     "count_items": 1, "count_pairs": 2, "count_gather": 1, "ellbar": 2,
                     "fft_rows": 1, "fft_cols": 1, "triple_fp32": 1, "triple_reduce": 1,
                     "normalise": 1, "check_triplets": 1, "tc_rows": 1, "triple_tc": 1}


def plan_kernels(n_grid, radius):
    tiles = -(-(n_grid - 1 + 2 * radius) // 16)
    passes = -(-int(tiles * tiles * 256).bit_length() // 11)   # keys: (tile, cell in the tile)
    return 1 + 2 * passes


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# DRAM traffic of one launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from the ncu captures summarised under profiles/, with the SHA-256 of the
# source file the kernel was built from when it was captured.  A kernel whose
# source has changed since then reports null.
MEASURED_TRAFFIC = {
    "grid": {"bytes": 20339968, "source": "paper_2412_02246_gb300/csrc/grid.cu",
           "sha256": "70be2b06c383f602aaf00e7804b1cc35bdaa232fc73ae16926d4d3499348f46e"},
    "fft_rows": {"bytes": 2880000, "source": "paper_2412_02246_gb300/csrc/fft.cu",
               "sha256": "eb38a2816f985ec629765661f3343c9580143cf0c7c03b76c4de5f6d4d3858b1"},
    "fft_cols": {"bytes": 722688, "source": "paper_2412_02246_gb300/csrc/fft.cu",
               "sha256": "eb38a2816f985ec629765661f3343c9580143cf0c7c03b76c4de5f6d4d3858b1"},
    "triple_fp32": {"bytes": 6663168, "source": "paper_2412_02246_gb300/csrc/triple.cu",
                  "sha256": "9a60a87aacafce2b1892ae57df49c65a93128134aa022893817ffe6aa540d175"},
    "triple_tc": {"bytes": 6703872, "source": "paper_2412_02246_gb300/csrc/triple_tc.cu",
                "sha256": "2366406142f503e351c2cf81f0169e8a6f3923eb458df2fbe972621d9f20abd3"},
    # one channel of the multi-channel workload (channel 0)
    "channel_fft_rows": {"bytes": 660686848, "source": "paper_2412_02246_gb300/csrc/fft.cu",
                         "sha256": "eb38a2816f985ec629765661f3343c9580143cf0c7c03b76c4de5f6d4d3858b1"},
    "channel_triple_tc": {"bytes": 829349120, "source": "paper_2412_02246_gb300/csrc/triple_tc.cu",
                          "sha256": "df4ad8e191f63240b08a8b4097b641d8d02e4da3c61b2ae31542aad2c465f3a9"},
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


def whole_job_rate(total_ms, steps, world, dev):
    """Whole-job estimates/s over all ranks: every rank ran `steps` independent
    replicas in `total_ms`; the job takes as long as its slowest rank (MAX over
    ranks), and the units are those of all ranks.  Returns (rate, max_ms)."""
    import torch
    t_max = float(total_ms)
    if world > 1:
        t = torch.tensor([t_max], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    return world * steps / (t_max * 1e-3), t_max


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


def uneven_batch(n_items, dev):
    """The first n_items of the seeded 256-item uneven batch, resident on the device."""
    import torch

    import paper_2412_02246_gb300 as absmod
    from paper_2412_02246_gb300 import synth
    rng = np.random.default_rng(2412)
    items = []
    for i in range(n_items):
        inp = synth.make_inputs(3, i, wl=synth.batch_item(rng, i))
        cfg = absmod.Config.from_workload(inp.wl)
        nt = len(absmod.abs_triplets(cfg))
        items.append((cfg, torch.from_numpy(inp.uv).to(dev),
                      torch.from_numpy(synth.vis_as_float2(inp.vis)).to(dev), nt, None,
                      torch.empty(nt, dtype=torch.float64, device=dev),
                      torch.empty(nt, dtype=torch.int64, device=dev),
                      torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)))
    return {"items": items}


def multichannel(args, m, synth, torch, dev, stream, peaks_sm):
    """The multi-channel workload: args.channels channels spread over 139-169 MHz (4096^2 grid,
    1e7 visibilities, 128 log rings, split-BF16), one abs_estimate_batched call over all of them,
    timed as channels/s; then each channel once more through abs_estimate with the stage profiler
    for the large-size rooflines (transforms, split-BF16 triplets, exact counts)."""
    if args.channels <= 0:
        return None
    wl = synth.workload(4)
    cfg = m.Config.from_workload(wl)
    ijk = m.abs_triplets(cfg)
    nt, N = len(ijk), m.abs_fft_size(cfg)
    nch = wl.extra["n_chan"]
    chans = sorted({int(round(x)) for x in np.linspace(0, nch - 1, args.channels)})
    ctx = m.Context(dev.index or 0, stream)
    items = []
    for ch in chans:
        inp = synth.channel_inputs(ch, wl=wl)
        items.append((cfg, torch.from_numpy(inp.uv).to(dev), torch.from_numpy(synth.vis_as_float2(inp.vis)).to(dev),
                      nt, None, torch.empty(nt, dtype=torch.float64, device=dev),
                      torch.empty(nt, dtype=torch.int64, device=dev),
                      torch.empty(cfg.n_bins, dtype=torch.float64, device=dev)))
    for _ in range(2):                         # eager (setups, workspaces), then graph capture
        ctx.abs_estimate_batched(items)
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        ctx.abs_estimate_batched(items)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    # per-channel stage times (eager, one channel at a time) and the work each stage did
    ctx.profile(True)
    visits = 0
    for it in items:
        ctx.abs_estimate(cfg, it[1], it[2], nt, None, *it[5:])
    torch.cuda.synchronize(dev)
    prof = ctx.profile_read()
    ctx.profile(False)
    n = cfg.n_grid
    q = m.abs_ring_q(cfg)
    mk = torch.empty((n, n), dtype=torch.uint8, device=dev)
    g = torch.empty((n, n, 2), dtype=torch.float32, device=dev)
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    fills = 0
    for it in items:
        ctx.abs_grid(cfg, it[1], it[2], g, w, mk)
        ctx.sync()
        A, F = ring_census(mk.cpu().numpy(), q, n)
        visits += count_route_visits(A, F)
        fills += int(F.sum())
    shape = ctx.tuned_shape(cfg)
    ctx.close()
    per = {k: 1e3 * v[0] / len(items) for k, v in prof.items()}   # us per channel
    rm = ring_rmax(q, n // 2 - 1)
    nb = cfg.n_bins
    lines = sum(2 * r + 1 for r in (max(rm[a], rm[a + 1] if a + 1 < nb else -1) for a in range(0, nb, 2)) if r >= 0)
    P = N * N
    hbm = load_peaks()
    kr = {}
    for i, j, k in ijk.tolist():
        lo, hi = kr.get((i, j), (1 << 30, -1))
        kr[(i, j)] = (min(lo, k), max(hi, k))
    by_j = sorted(kr, key=lambda ij: (ij[1], ij[0]))
    band = 0
    for t in range(0, len(by_j), 128):
        tile = by_j[t:t + 128]
        band += -(-(max(kr[r][1] for r in tile) - min(kr[r][0] for r in tile) + 1) // 16) * 16
    out = {"value": len(items) * 1e3 / ms, "unit": "channels/s", "channels": chans,
           "ms_per_call": ms, "n_trip": nt, "n_fft": N, "tc_shape": shape,
           "stages_us_per_channel": {k: round(v, 1) for k, v in sorted(per.items())}}

    def frac(ach, peak):
        return {"achieved": ach, "peak": peak, "frac": ach / peak}
    if "fft_rows" in per:
        out["fft_rows"] = dict(frac((lines * N * 8 + nb * P * 4) / (per["fft_rows"] * 1e-6) / 1e9,
                                    hbm["hbm_gbs"]), bound="hbm", unit="GB/s",
                               traffic=measured_traffic("channel_fft_rows"))
    if "fft_cols" in per:
        out["fft_cols"] = dict(frac((fills * 24 / len(items) + lines * N * 8) / (per["fft_cols"] * 1e-6) / 1e9,
                                    hbm["hbm_gbs"]), bound="hbm", unit="GB/s")
    if "triple_tc" in per:
        out["triple_tc"] = dict(frac(2.0 * 128 * 3 * band * P / (per["triple_tc"] * 1e-6) / 1e12,
                                     hbm["bf16_tflops"]), bound="tensor", unit="TFLOP/s",
                                useful_tflops=2.0 * nt * P / (per["triple_tc"] * 1e-6) / 1e12,
                                traffic=measured_traffic("channel_triple_tc"))
    if "count_pairs" in per:
        out["count_pairs"] = {"pair_visits_per_channel": visits // len(items),
                              "gvisits_per_s": visits / len(items) / (per["count_pairs"] * 1e-6) / 1e9}
    out["note"] = ("4096^2 grid, 1e7 visibilities, 128 log rings over l 46-1320, split-BF16, one baseline set "
                   "scaled by frequency; value = channels / device time of one abs_estimate_batched call "
                   "(inputs resident); stage times from one eager abs_estimate per channel")
    return out


def roofline_for(stage, avg_ms, geo, peaks):
    """Algorithmic work of one launch of `stage` over its average duration.

    grid:        FP32 lane-ops, 4 per (visibility, footprint cell): w = wx wy, two FMAs, one add
    count_pairs: integer pair visits (of the route the kernel takes) x 2 lane-ops (index add, ring
                 compare); a grid with no holes takes the holes route with no visits at all
    triple_fp32: 2 flops per (triplet, pixel)
    triple_tc:   executed BF16 tensor flops: per 128-row tile 2 M N K with M = 128, N = 3 x its ring
                 band (the stacked [Bh; Bl] MMA and the Al Bh MMA), K = pixels
    fft_rows/cols, others: algorithmic bytes (reads + writes of the data the kernel must move)
    """
    s = avg_ms * 1e-3
    lane_ops = geo["sm"] * 128 * geo["clk_hz"]
    out = {}
    if stage == "grid":
        ops = 4.0 * geo["n_vis"] * geo["footprint"]
        out = {"bound": "alu", "achieved": ops / s / 1e12, "peak": lane_ops / 1e12, "unit": "Tlane-op/s"}
    elif stage == "count_pairs":
        ops = 2.0 * geo["pair_visits"]
        out = {"bound": "alu", "achieved": ops / s / 1e12, "peak": lane_ops / 1e12, "unit": "Tlane-op/s",
               "pair_visits": geo["pair_visits"]}
    elif stage == "triple_fp32":
        fl = 2.0 * geo["n_trip"] * geo["P"]
        out = {"bound": "alu", "achieved": fl / s / 1e12, "peak": 2 * lane_ops / 1e12, "unit": "TFLOP/s"}
    elif stage == "triple_tc":
        fl = 2.0 * 128 * 3 * geo["tc_band_sum"] * geo["P"]
        out = {"bound": "tensor", "achieved": fl / s / 1e12, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s"}
    else:
        byts = geo["bytes"].get(stage)
        if byts is None:
            return {"bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": None,
                    "traffic": measured_traffic(stage)}
        out = {"bound": "hbm", "achieved": byts / s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    out["frac"] = out["achieved"] / out["peak"]
    out["traffic"] = measured_traffic(stage)
    return out


def workload_geometry(m, cfg, ctx, uv, vis, ijk, N, wl, dev, torch):
    """Counts that the roofline needs: filled ring cells (pair visits), padded tiles, bytes."""
    n = cfg.n_grid
    g = torch.empty((n, n, 2), dtype=torch.float32, device=dev)
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    mk = torch.empty((n, n), dtype=torch.uint8, device=dev)
    ctx.abs_grid(cfg, uv, vis, g, w, mk)
    ctx.sync()
    mask = mk.cpu().numpy()
    q = m.abs_ring_q(cfg)
    A, c = ring_census(mask, q, n)
    visits = count_route_visits(A, c)
    # the split-BF16 kernel's row tiles: rows by (j, i), 128 a tile, each with its band of k rounded to 16
    kr = {}
    for i, j, kk in ijk:
        lo, hi = kr.get((int(i), int(j)), (1 << 30, -1))
        kr[(int(i), int(j))] = (min(lo, int(kk)), max(hi, int(kk)))
    by_j = sorted(kr, key=lambda ij: (ij[1], ij[0]))
    band_sum = 0
    for t in range(0, len(by_j), 128):
        tile = by_j[t:t + 128]
        lo = min(kr[r][0] for r in tile)
        hi = max(kr[r][1] for r in tile)
        band_sum += -(-(hi - lo + 1) // 16) * 16
    nb = cfg.n_bins
    P = N * N
    # transforms: the column pass reads the ring cells' FP64 sums (re, im, w) and writes
    # 2 R_pair + 1 transformed columns of N points per ring pair; the row pass reads them
    # back and writes every field.  Points are double-float complex (16 B) on the FP32
    # path, FP32 complex (8 B) on the split-BF16 path.
    rm = ring_rmax(q, n // 2 - 1)
    lines = sum(2 * max(rm[a], rm[a + 1] if a + 1 < nb else -1) + 1 for a in range(0, nb, 2)
                if max(rm[a], rm[a + 1] if a + 1 < nb else -1) >= 0)
    pt = 8 if cfg.precision == m.ABS_SPLIT_BF16 else 16
    fft_cols_bytes = int(c.sum()) * 24 + lines * N * pt
    fft_rows_bytes = lines * N * pt + nb * P * 4
    return {"pair_visits": int(visits), "n_trip": len(ijk), "P": P, "n_vis": len(uv),
            "footprint": (2 * cfg.radius_cells + 1) ** 2,
            "tc_band_sum": band_sum,
            "bytes": {"fft_rows": fft_rows_bytes, "fft_cols": fft_cols_bytes,
                      "ring_lists": n * n * 2}}


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
    # a stream of our own (the library captures CUDA graphs on it; the legacy
    # default stream cannot be captured)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    uv = torch.from_numpy(inp.uv).to(dev)
    vis = torch.from_numpy(synth.vis_as_float2(inp.vis)).to(dev)
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
    # timed region: the production path (stage profiler off, so abs_estimate
    # replays its captured CUDA graph)
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
    # per-stage device times: the same steps again with the CUDA-event stage
    # profiler on (eager launches, events on the launching stream)
    ctx.profile(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        step()
    torch.cuda.synchronize(dev)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.sync()
    value, t_max = whole_job_rate(total_ms, args.steps, world, dev)

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
    # results layer over the batch: (l1, mu, t) cells (5 x 5 shape bins) and ensemble mean / spread
    cells = [torch.empty((cfg.n_bins, 5, 5), dtype=torch.float64, device=dev) for _ in range(3)]
    ctx.abs_rebin(cfg, BR, T, E, None, 5, 5, *cells)
    e0.record(stream)
    for _ in range(reps):
        ctx.abs_rebin(cfg, BR, T, E, None, 5, 5, *cells)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    rebin_us = 1e3 * e0.elapsed_time(e1) / reps

    # uneven batch: independent items of different grid sizes, rings and precisions in one call
    uneven = None
    if args.batch_items > 0:
        bi = uneven_batch(args.batch_items, dev)
        for _ in range(2):                     # eager (setups, workspaces), then graph capture
            ctx.abs_estimate_batched(bi["items"])
        ctx.sync()
        reps_u = max(1, args.steps // 10)
        e0.record(stream)
        for _ in range(reps_u):
            ctx.abs_estimate_batched(bi["items"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        uneven = len(bi["items"]) * reps_u / (e0.elapsed_time(e1) * 1e-3)
        del bi

    # visibility simulator (Eqs. beam, vis): 10^5 of the workload's baselines, a 256^2 map of the
    # paper's 0.029 deg pixels times the MWA tile beam, direct DFT
    msim, nsim = 256, 100_000
    simulator, chan = None, None
    if rank == 0:   # the sections below are outside the timed region: rank 0 alone runs them
        sky = torch.from_numpy(synth.quadratic_sky(synth.gaussian_field(msim, np.random.default_rng(5)), 0.3)
                               .astype(np.float32)).to(dev)
        vsim = torch.empty((nsim, 2), dtype=torch.float32, device=dev)
        dth = float(np.deg2rad(0.029))
        d_over_lam = 4.0 / (299792458.0 / 154.25e6)
        ctx.abs_simulate_vis(sky, dth, uv[:nsim], vsim, m.ABS_BEAM_MWA_TILE, d_over_lam)
        e0.record(stream)
        ctx.abs_simulate_vis(sky, dth, uv[:nsim], vsim, m.ABS_BEAM_MWA_TILE, d_over_lam)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sim_s = e0.elapsed_time(e1) * 1e-3
        simulator = {"vis_per_s": nsim / sim_s, "phase_terms_per_s": nsim * msim * msim / sim_s,
                     "ms": sim_s * 1e3, "n_vis": nsim, "map": msim,
                     "note": "abs_simulate_vis: MWA tile beam, 0.029 deg pixels, direct DFT (double-float "
                             "phase and SFU sincos every 16 pixels, complex rotation between)"}
        del sky, vsim
        # (an NVTX range, so that a profiler can select this section's launches)
        torch.cuda.nvtx.range_push("multichannel")
        chan = multichannel(args, m, synth, torch, dev, stream,
                            peaks_sm=torch.cuda.get_device_properties(dev).multi_processor_count)
        torch.cuda.nvtx.range_pop()

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

    # split-BF16 (tcgen05) form on the same workload and GPU
    cfg_tc = m.Config.from_workload(wl, precision=m.ABS_SPLIT_BF16)
    for _ in range(args.warmup):
        flush.fill_(1.0)
        ctx.abs_estimate(cfg_tc, uv, vis, nt, None, B, T, E)
    ctx.sync()
    ev_tc = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev_tc[k][0].record(stream)
        ctx.abs_estimate(cfg_tc, uv, vis, nt, None, B, T, E)
        ev_tc[k][1].record(stream)
    torch.cuda.synchronize(dev)
    tc_ms = sum(a.elapsed_time(b) for a, b in ev_tc)
    ctx.profile(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        ctx.abs_estimate(cfg_tc, uv, vis, nt, None, B, T, E)
    torch.cuda.synchronize(dev)
    prof_tc = ctx.profile_read()
    ctx.profile(False)

    # per-kernel averages and the dominant kernel's roofline
    stages = {k: {"ms_total": v[0], "launches": v[1], "avg_us": 1e3 * v[0] / max(v[1], 1)}
              for k, v in prof.items()}
    kps = dict(KERNELS_PER_STAGE, grid_plan=plan_kernels(wl.n_grid, wl.radius_cells))
    launches = sum(kps.get(k, 1) * v[1] for k, v in prof.items())
    # the dominant kernel: the single-kernel stage with the most device time
    dom = max(((k, v) for k, v in prof.items() if kps.get(k, 1) == 1), key=lambda kv: kv[1][0])[0]
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or 1900.0
    geo = workload_geometry(m, cfg, ctx, uv, vis, ijk, N, wl, dev, torch)
    geo["sm"] = props.multi_processor_count
    geo["clk_hz"] = sm_mhz * 1e6
    roof = roofline_for(dom, stages[dom]["avg_us"] * 1e-3, geo, peaks)
    roof["kernel"] = dom
    roof["peak_source"] = peaks["source"]
    other_roofs = {}
    for k in ("grid", "fft_rows", "fft_cols", "count_pairs", "triple_fp32"):
        if k in stages and k != dom:
            rr = roofline_for(k, stages[k]["avg_us"] * 1e-3, geo, peaks)
            other_roofs[k] = {kk: rr[kk] for kk in ("bound", "achieved", "peak", "unit", "frac", "traffic",
                                                    "pair_visits") if kk in rr}
    tri_fp32 = roofline_for("triple_fp32", stages["triple_fp32"]["avg_us"] * 1e-3, geo, peaks)
    tc_avg = 1e3 * prof_tc["triple_tc"][0] / max(prof_tc["triple_tc"][1], 1)
    tc_shape = ctx.tuned_shape(cfg_tc)      # the autotuner's pick (chunk width, grouped tiles)
    tri_tc = roofline_for("triple_tc", tc_avg * 1e-3, geo, peaks)
    useful = 2.0 * nt * N * N

    cpu_s = oracle_estimate_seconds(inp)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wl), "clocks": clk,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches), "roofline": roof, "stage_rooflines": other_roofs,
        "cpu_baseline": {"value": 1.0 / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one full realisation of the workload (plain C FP64, brute-force "
                                   "closed-triangle sums)"},
        "batched": {"value": batched, "unit": UNIT, "realisations_per_call": R,
                    "rebin_us": round(rebin_us, 2),
                    "note": "abs_estimate_many: realisations sharing one baseline set (plan, counts "
                            "and ring tables once per call)"},
        "batched_uneven": {"value": uneven, "unit": UNIT, "items_per_call": args.batch_items,
                           "note": "abs_estimate_batched: independent items, grid {256,512,1024}^2, "
                                   "1e5-1e6 visibilities, 16-48 log l bins, split-BF16 triplets, one CUDA "
                                   "graph per call; seeded item shapes, the first items_per_call of the "
                                   "256-item batch"},
        "split_bf16": {"value": args.steps / (tc_ms * 1e-3), "unit": UNIT,
                       "triple_tc_us": round(tc_avg, 2),
                       "tc_shape": tc_shape,
                       "triple_tc_tflops_executed": tri_tc["achieved"],
                       "triple_tc_frac_bf16_peak": tri_tc["frac"],
                       "triple_tc_traffic": tri_tc["traffic"],
                       "triple_useful_tflops": useful / (tc_avg * 1e-6) / 1e12},
        "multichannel": chan,
        "simulator": simulator,
        "fp32": {"triple_fp32_us": round(stages["triple_fp32"]["avg_us"], 2),
                 "triple_useful_tflops": useful / (stages["triple_fp32"]["avg_us"] * 1e-6) / 1e12,
                 "frac_fp32_simt_peak": tri_fp32["frac"]},
        "stages_us": {k: round(v["avg_us"], 2) for k, v in sorted(stages.items())},
        "kernel_timing": "stage device times: CUDA events around each stage on the library's stream, "
                         "in a second pass of the same steps with graphs off",
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
    ap.add_argument("--batch-items", type=int, default=64, help="items of the uneven batch (0: skip it)")
    ap.add_argument("--channels", type=int, default=8,
                    help="channels of the multi-channel workload, spread over the band (0: skip it)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
