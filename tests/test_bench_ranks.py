"""The multi-rank (replica) logic of bench.py on CPU with the gloo backend,
world size 2: the timed region is the slowest rank's, every rank learns it, and
the reported value is the whole job's rate; the reference arm runs on rank 0
only (other ranks exit 0 without work or output)."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank                     # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    out.put((rank, ms, bench.replica_rate(20, 16, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_rate_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(ms == 150.0 for _, ms, _ in res)              # both ranks see the slowest time
    assert all(v == pytest.approx(20 * 16 * 2 / 0.150) for _, _, v in res)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.replica_rate(10, 1, 1, 20.0) == pytest.approx(500.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
