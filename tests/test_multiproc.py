"""Multi-rank path of bench.py on the CPU (gloo, world size 2): the estimator
does not shard, so N GPUs run N independent replicas; the whole-job rate is
the units of all ranks over the slowest rank's time.  No GPU is used."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank 1 is the slow one: 400 ms for 10 steps, rank 0 250 ms
    rate, t_max = bench.whole_job_rate(250.0 if rank == 0 else 400.0, 10, world, torch.device("cpu"))
    q.put((rank, rate, t_max))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, t_max in got:
        assert t_max == 400.0                       # MAX over ranks
        assert abs(rate - 2 * 10 / 0.4) < 1e-9      # both ranks' units over the slowest time


def test_whole_job_rate_single_rank():
    import bench
    rate, t_max = bench.whole_job_rate(200.0, 20, 1, torch.device("cpu"))
    assert t_max == 200.0 and abs(rate - 100.0) < 1e-9


def test_replicas_share_baselines_but_not_skies():
    """Each rank's replica observes the same array with its own sky realisation."""
    from paper_2412_02246_gb300 import synth
    a, b = synth.make_inputs(0, 0), synth.make_inputs(0, 1)
    assert (a.uv == b.uv).all()
    assert not (a.vis == b.vis).all()


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
