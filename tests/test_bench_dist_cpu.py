"""The N > 1 path of bench.py on CPU: two gloo ranks, each an independent
replica, combine their timings with a barrier and a max-over-ranks all-reduce
(no data-path collective).  Checks the max and the whole-job throughput."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        elapsed = 100.0 + 50.0 * rank             # the second replica is slower
        mx = bench.max_over_ranks(elapsed, world, device="cpu")
        v = bench.job_throughput(world, 3, 8.0 * 4096 ** 3 / 3, mx)
        q.put((rank, mx, v))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [150.0, 150.0]
    expect = 2 * 3 * (8.0 * 4096 ** 3 / 3) / 0.150 / 1e9
    assert all(abs(o[2] - expect) < 1e-6 * expect for o in out)
