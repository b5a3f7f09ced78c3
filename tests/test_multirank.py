"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU).  Each
rank times its own replica; rank 0 reports every rank's units over the
slowest rank's time."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    times = [10.0 + 5.0 * rank, 3.0 - rank, 7.5]  # per-rank step, instrumented, e2e times (ms)
    got = bench.max_over_ranks(times, w)
    out[rank] = (r, w, local, got, bench.whole_job_rate(1000, w, got[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        rr, w, local, got, rate = res[r]
        assert (rr, w, local) == (r, 2, r)
        assert got == [15.0, 3.0, 7.5]
        assert rate == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_is_identity():
    assert bench.max_over_ranks([1.5, 2.0], 1) == [1.5, 2.0]
    assert bench.whole_job_rate(500, 1, 250.0) == pytest.approx(2000.0)
