"""The multi-process path of bench.py on CPU (gloo, two ranks): the timed quantities
are reduced to the slowest rank's on every rank, and the whole-job rate counts every
rank's replica.  (Every run here has one GPU; the replicas share no data, so this host
logic is the whole of the N > 1 path.)"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = [12.5, 17.25][rank]          # this rank's timed milliseconds
    got = bench.max_over_ranks(mine, world, "cpu")
    e2e = bench.max_over_ranks(0.5 + rank, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, e2e))


def test_two_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [17.25, 17.25]
    assert [r[2] for r in res] == [1.5, 1.5]


def test_job_rate_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench

    one = bench.job_mlups(2048 * 512, 200, 1, 0.011)
    two = bench.job_mlups(2048 * 512, 200, 2, 0.011)
    assert two == pytest.approx(2 * one)
    assert one == pytest.approx(2048 * 512 * 200 / 0.011 / 1e6)
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
