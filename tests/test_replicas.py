"""Multi-rank host logic of the benchmark (replicas: one measurement per rank, no exchange of data):
two gloo ranks on the CPU exchange their timings through the same collectives the benchmark uses."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    barrier, max_over_ranks = bench.rank_collectives(world, "cpu")
    barrier()
    ms = 10.0 + 5.0 * rank                     # the slower rank decides
    m = max_over_ranks(ms)
    out[rank] = (m, bench.replica_throughput(world, 3, m / 1e3))
    barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    m, thr = res[0]
    assert m == 15.0
    assert thr == pytest.approx(2 * 3 / 0.015)
