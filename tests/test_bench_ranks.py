"""The multi-GPU form of bench.py shards whole images across ranks (weak
scaling, no data-path collective) and reports the slowest rank's time: its
host logic, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    d = bench.init_dist(ws, "gloo")
    ms_local = 10.0 + 5.0 * r                    # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, d)
    seeds = bench.image_seeds(r, 4)
    value = bench.job_value(2 * 4 * 100, ws, ms)
    q.put((r, ms, seeds, value))
    d.barrier()
    d.destroy_process_group()


def test_two_gloo_ranks_shard_images_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert all(ms == 15.0 for _, ms, _, _ in out)            # max over ranks
    s0, s1 = set(out[0][2]), set(out[1][2])
    assert not (s0 & s1) and len(s0) == len(s1) == 4         # disjoint images
    assert out[0][3] == out[1][3] == pytest.approx(2 * 4 * 100 * 2 / 15e-3)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(3.0, None) == 3.0
