"""The multi-rank logic of bench.py on CPU: two gloo ranks (replicas, weak scaling)."""
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


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed (r + 1) * 1000 units in 10 + r ms
        units, ms = bench.reduce_over_ranks((rank + 1) * 1000, 10.0 + rank)
        p = bench.make_problem(rank, 128)
        q.put((rank, units, ms, float(p.y[:8].sum()), p.m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_units_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, units, ms, _, _ in out:
        assert units == 3000.0 and ms == 11.0, rank
    # every rank solves its own instance (its own seed): replicas, no shared data
    assert out[0][3] != out[1][3]
    assert out[0][4] == out[1][4]


def test_single_rank_without_process_group_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(123, 4.5) == (123.0, 4.5)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
