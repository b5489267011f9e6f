"""The benchmark's multi-rank logic on CPU with the gloo backend (world size
2): the job time is the slowest rank's, the throughput counts every rank's
cells (weak scaling, no collective on the data path), and the reference arm
runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 10.0 + 5.0 * rank
    got = bench.max_over_ranks(mine)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 15.0, 1: 15.0}


def test_weak_value_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.weak_value(1, 10000, 20, 6.0)
    two = bench.weak_value(2, 10000, 20, 6.0)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(10000 * 20 / 6e-3)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_lockstep_waste_definition():
    sys.path.insert(0, ROOT)
    import bench
    # pairs (3, 5) and (4, 4): the first pair idles 2 lane-iterations of 16 useful
    assert bench.lockstep_waste([3, 5, 4, 4], 2) == pytest.approx(2 / 16)
    assert bench.lockstep_waste([7] * 6, 2) == 0.0
    assert bench.lockstep_waste([2, 6, 1], 2) == pytest.approx((4 + 1) / 9)
