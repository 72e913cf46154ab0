"""Checkpoint / resume for long batched runs (harness level).

``run_resumable`` runs ``abs_estimate_batched`` over the items whose results
are not yet on disk, a chunk at a time, and writes each finished item's
(B, counts, ellbar) to ``<out_dir>/<name>.npz`` atomically (a temporary file,
then a rename), so a run that is interrupted can be started again and skips
what is done.  The estimates themselves run in the library's kernels; this
module only decides which items to submit and stores their outputs.
"""
from __future__ import annotations

import os

import numpy as np


def _done(out_dir: str, name: str) -> bool:
    return os.path.exists(os.path.join(out_dir, name + ".npz"))


def run_resumable(ctx, items, names, out_dir: str, chunk: int = 16) -> list:
    """items: tuples as Context.abs_estimate_batched takes them, (cfg, uv, vis, n_trip, ijk,
    B, counts, ellbar) with device tensors; names: one unique file stem per item.
    Returns the names run by this call (the others were already on disk)."""
    if len(names) != len(items) or len(set(names)) != len(names):
        raise ValueError("one unique name per item is required")
    os.makedirs(out_dir, exist_ok=True)
    todo = [k for k, nm in enumerate(names) if not _done(out_dir, nm)]
    ran = []
    for c0 in range(0, len(todo), max(1, chunk)):
        part = todo[c0:c0 + max(1, chunk)]
        ctx.abs_estimate_batched([items[k] for k in part])
        ctx.sync()
        for k in part:
            B, counts, ellbar = items[k][5], items[k][6], items[k][7]
            final = os.path.join(out_dir, names[k] + ".npz")
            tmp = final + ".tmp.npz"
            np.savez(tmp, B=B.cpu().numpy(), counts=counts.cpu().numpy(), ellbar=ellbar.cpu().numpy())
            os.replace(tmp, final)
            ran.append(names[k])
    return ran


def load_result(out_dir: str, name: str) -> dict:
    with np.load(os.path.join(out_dir, name + ".npz")) as z:
        return {k: z[k] for k in z.files}
