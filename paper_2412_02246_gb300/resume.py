"""Checkpoint / resume for long batched runs (harness level).

``run_resumable`` runs ``abs_estimate_batched`` over the items whose results
are not yet on disk, a chunk at a time, and writes each finished item's
(B, counts, ellbar) to ``<out_dir>/<name>.npz``: to a temporary file that is
flushed to disk (fsync) and then renamed over the final name (the directory
is fsynced too), so a run that is interrupted, even by a power loss, can be
started again and skips what is done.  Each file carries a fingerprint of
the item's setup (configuration, visibility count, triplet count and an
optional caller tag such as the input's seed); a file whose fingerprint does
not match the item is not taken as done, and the item runs again.  The
estimates themselves run in the library's kernels; this module only decides
which items to submit and stores their outputs.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np


def fingerprint(item, tag: str = "") -> str:
    """Hex digest of what determines an item's result besides its data: the
    configuration's fields, n_vis, n_trip and the caller's tag."""
    cfg, uv, _, n_trip = item[0], item[1], item[2], item[3]
    parts = []
    if cfg is not None:
        for f in ("n_grid", "du", "kernel", "sigma_cells", "radius_cells", "n_fft", "precision", "norm_A",
                  "weight_mode"):
            parts.append(f"{f}={getattr(cfg, f, None)!r}")
        parts.append("edges=" + np.asarray(cfg.ell_edges, np.float64).tobytes().hex())
    n_vis = uv.shape[0] if hasattr(uv, "shape") else uv
    parts += [f"n_vis={n_vis}", f"n_trip={int(n_trip)}", f"tag={tag}"]
    return hashlib.sha256("|".join(parts).encode()).hexdigest()


def _done(out_dir: str, name: str, fp: str) -> bool:
    path = os.path.join(out_dir, name + ".npz")
    if not os.path.exists(path):
        return False
    try:
        with np.load(path) as z:
            return "fingerprint" in z.files and str(z["fingerprint"]) == fp
    except (OSError, ValueError):
        return False


def _write_synced(final: str, **arrays):
    tmp = final + ".tmp.npz"
    with open(tmp, "wb") as fh:
        np.savez(fh, **arrays)
        fh.flush()
        os.fsync(fh.fileno())
    os.replace(tmp, final)
    dfd = os.open(os.path.dirname(final) or ".", os.O_RDONLY)
    try:
        os.fsync(dfd)
    finally:
        os.close(dfd)


def run_resumable(ctx, items, names, out_dir: str, chunk: int = 16, tags=None) -> list:
    """items: tuples as Context.abs_estimate_batched takes them, (cfg, uv, vis, n_trip, ijk,
    B, counts, ellbar) with device tensors; names: one unique file stem per item; tags:
    optional per-item strings (e.g. the seed of its inputs) folded into the fingerprint.
    Returns the names run by this call (the others were already on disk with a
    matching fingerprint)."""
    if len(names) != len(items) or len(set(names)) != len(names):
        raise ValueError("one unique name per item is required")
    if tags is not None and len(tags) != len(items):
        raise ValueError("one tag per item is required")
    os.makedirs(out_dir, exist_ok=True)
    fps = [fingerprint(it, "" if tags is None else str(tags[k])) for k, it in enumerate(items)]
    todo = [k for k, nm in enumerate(names) if not _done(out_dir, nm, fps[k])]
    ran = []
    for c0 in range(0, len(todo), max(1, chunk)):
        part = todo[c0:c0 + max(1, chunk)]
        ctx.abs_estimate_batched([items[k] for k in part])
        ctx.sync()
        for k in part:
            B, counts, ellbar = items[k][5], items[k][6], items[k][7]
            _write_synced(os.path.join(out_dir, names[k] + ".npz"), B=B.cpu().numpy(),
                          counts=counts.cpu().numpy(), ellbar=ellbar.cpu().numpy(),
                          fingerprint=np.array(fps[k]))
            ran.append(names[k])
    return ran


def load_result(out_dir: str, name: str) -> dict:
    with np.load(os.path.join(out_dir, name + ".npz")) as z:
        return {k: z[k] for k in z.files}
