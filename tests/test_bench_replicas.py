"""The multi-rank path of bench.py on the CPU: two gloo ranks run the same
host-side logic the GPU replicas use (rank and world from the environment,
the job's time as the slowest rank's, whole-job throughput over all ranks).
The fixed-rank path has no exchange step, so replicas share nothing else."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    w, r, loc = bench.dist_setup(None)
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        value = bench.replica_throughput(w, 5, ms)
        dist.barrier()
    finally:
        dist.destroy_process_group()
    q.put((rank, w, r, loc, ms, value))


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, w, r, loc, ms, value in res:
        assert (w, r, loc) == (2, rank, rank)
        assert ms == 20.0                          # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 5 / 0.020)  # both ranks' units over that time


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.replica_throughput(1, 30, 1000.0) == pytest.approx(30.0)
