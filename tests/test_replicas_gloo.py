"""The multi-rank bench path on CPU (world size 2, gloo): replicas share no data-path
collective; the job time is the slowest rank's and the throughput counts every rank's
eigenpairs (weak scaling)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [1200.0, 1500.0]                 # per-rank summed step times (ms)
    t = bench.max_over_ranks(times[rank], world, "cpu")
    out[rank] = (t, bench.replica_throughput(world, 12, 5, t))
    dist.destroy_process_group()


def test_two_replicas_report_slowest_rank_and_job_throughput():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, v = res[0]
    assert t == 1500.0
    assert v == pytest.approx(2 * 12 * 5 / 1.5)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.replica_throughput(1, 8, 2, 1000.0) == pytest.approx(16.0)
