"""The host logic of bench.py for several GPUs (one process per GPU, replicas
only): every rank times its own system, the job time is the slowest rank's,
and the rate counts the atoms of all ranks.  Run as two gloo processes on the
CPU (no GPU, no CUDA call)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, secs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(dist, secs[rank], device="cpu")
        out[rank] = (m, bench.whole_job_rate(world, 1000, 50, m))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_atoms():
    world = 2
    secs = [0.5, 2.0]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, _free_port_once(), secs, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        got = dict(out)
    for r in range(world):
        m, rate = got[r]
        assert m == pytest.approx(2.0)
        assert rate == pytest.approx(world * 1000 * 50 / 2.0)


_PORT = None


def _free_port_once():
    global _PORT
    if _PORT is None:
        _PORT = _free_port()
    return _PORT


def test_single_process_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(None, 1.25) == 1.25
    assert bench.whole_job_rate(1, 1_000_000, 1000, 0.5) == pytest.approx(2.0e9)
