"""CPU: the multi-GPU bench's host logic under torch.distributed (gloo, two
ranks): block sharding covers every block once, and the timed region's
duration is the max over ranks.  Blocks are independent, so this reduction is
the only collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = bench.shard_blocks(4097, rank, world)
        t = bench.reduce_max(10.0 + 5.0 * rank)
        g = bench.whole_job_gbs(1 << 20, 4, t, world)
        q.put((rank, lo, hi, t, g))
    finally:
        dist.destroy_process_group()


def test_two_rank_shard_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, lo0, hi0, t0, g0), (r1, lo1, hi1, t1, g1) = res
    assert (lo0, hi0, lo1, hi1) == (0, 2049, 2049, 4097)      # contiguous, disjoint, complete
    assert t0 == t1 == 15.0                                      # the slowest rank's time
    assert g0 == g1 == pytest.approx(2 * (1 << 20) * 4 / 0.015 / 1e9)


def test_single_process_passthrough():
    assert bench.reduce_max(3.5) == 3.5
    assert bench.shard_blocks(10, 0, 1) == (0, 10)
