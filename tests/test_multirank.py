"""Host logic of the multi-rank benchmark on CPU: two gloo ranks, each with its
own box (no data-path exchange), time reduced by MAX, whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]
        m = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (m, bench.job_rate(1000, 4, 10, world, m))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_rate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        m, rate = out[r]
        assert m == 150.0
        assert rate == pytest.approx(2 * 1000 * 4 * 10 / 0.150)


def test_single_process_rate():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(8, 4, 2, 1, 1000.0) == pytest.approx(64.0)
