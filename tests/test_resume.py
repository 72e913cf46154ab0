"""Checkpoint / resume of batched runs (harness level, no GPU): an interrupted
run leaves the finished items on disk, and the rerun submits only the rest."""
import numpy as np
import pytest
import torch

from paper_2412_02246_gb300 import resume


class FakeCtx:
    """Stands in for Context: fills each item's outputs from its own index, and can
    fail on a chosen call (an interruption)."""

    def __init__(self, fail_on_call=None):
        self.calls, self.seen, self.fail_on_call = 0, [], fail_on_call

    def abs_estimate_batched(self, items):
        self.calls += 1
        if self.fail_on_call == self.calls:
            raise RuntimeError("interrupted")
        for it in items:
            tag = it[1]
            self.seen.append(tag)
            it[5].fill_(float(tag))
            it[6].fill_(tag)
            it[7].fill_(-float(tag))

    def sync(self):
        pass


def _items(n):
    return [(None, k, None, 4, None, torch.zeros(4, dtype=torch.float64), torch.zeros(4, dtype=torch.int64),
             torch.zeros(3, dtype=torch.float64)) for k in range(n)]


def test_interrupted_run_resumes_where_it_stopped(tmp_path):
    names = [f"item{k:03d}" for k in range(10)]
    with pytest.raises(RuntimeError):
        resume.run_resumable(FakeCtx(fail_on_call=3), _items(10), names, str(tmp_path), chunk=3)
    done = sorted(p.stem for p in tmp_path.glob("*.npz") if not p.name.endswith(".tmp.npz"))
    assert done == names[:6]                        # two chunks finished before the failure
    ctx = FakeCtx()
    ran = resume.run_resumable(ctx, _items(10), names, str(tmp_path), chunk=3)
    assert ran == names[6:] and ctx.seen == list(range(6, 10))
    for k, nm in enumerate(names):
        r = resume.load_result(str(tmp_path), nm)
        assert np.all(r["B"] == k) and np.all(r["counts"] == k) and np.all(r["ellbar"] == -k)
    assert resume.run_resumable(FakeCtx(), _items(10), names, str(tmp_path)) == []


def test_names_must_be_unique(tmp_path):
    with pytest.raises(ValueError):
        resume.run_resumable(FakeCtx(), _items(2), ["a", "a"], str(tmp_path))


def test_stale_results_of_another_setup_are_rerun(tmp_path):
    """A result on disk from a different setup (here another triplet count, then
    another caller tag) does not count as done."""
    names = [f"item{k}" for k in range(3)]
    resume.run_resumable(FakeCtx(), _items(3), names, str(tmp_path), tags=["s0", "s1", "s2"])
    ctx = FakeCtx()
    changed = _items(3)
    changed[1] = changed[1][:3] + (5,) + changed[1][4:]
    assert resume.run_resumable(ctx, changed, names, str(tmp_path), tags=["s0", "s1", "s2"]) == ["item1"]
    ctx = FakeCtx()
    assert resume.run_resumable(ctx, changed, names, str(tmp_path), tags=["s0", "s1", "x"]) == ["item2"]
    assert resume.run_resumable(FakeCtx(), changed, names, str(tmp_path), tags=["s0", "s1", "x"]) == []
