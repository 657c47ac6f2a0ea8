"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The selected inversion does not shard (every supernode reads all of its
ancestors), so several GPUs run independent replicas; the only cross-rank
step is the timing reduction (max over ranks) and the whole-job rate.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_info()
        assert (r, w, lr) == (rank, world, rank)
        local_ms = 10.0 + 5.0 * rank                    # rank 1 is the slow one
        mx = bench.reduce_max_over_ranks(local_ms)
        rate = bench.whole_job_rate(100.0, world, mx)
        out[rank] = (mx, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        mx, rate = out[r]
        assert mx == 15.0                               # the slowest rank's time
        assert rate == pytest.approx(2 * 100.0 / 15e-3)


def test_single_process_needs_no_group():
    import bench
    assert bench.reduce_max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
