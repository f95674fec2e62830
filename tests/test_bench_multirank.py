"""bench.py's multi-GPU path is replicas only: every rank times its own replica
between barriers and rank 0 reports the slowest rank's time.  The host side of
that path (process group, barrier, max over ranks, whole-job throughput) runs
here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), TLBM_BENCH_BACKEND="gloo")
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    r, ws, local = bench.dist_setup()
    assert (r, ws, local) == (rank, world, rank)
    bench.barrier(ws)
    slowest = bench.max_over_ranks(times[rank], ws)
    bench.barrier(ws)
    out[rank] = slowest
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    times = [1.25, 2.5]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.5
    # whole-job throughput of N replicas: N * units / slowest time
    units, steps = 67125249, 100
    assert 2 * units * steps / out[0] / 1e9 == pytest.approx(2 * units * steps / 2.5 / 1e9)


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench

    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.dist_setup() == (0, 1, 0)
    assert bench.max_over_ranks(3.0, 1) == 3.0
