"""The replica timing of bench.py (--gpus N): the slowest rank sets the time and
the whole-job rate counts every replica's steps.  Two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks([1.0 + rank, 10.0 * (rank + 1), 5.0 - rank], world)
    out[rank] = (got, bench.replica_rate(world, 10, got[1]))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, rate = res[r]
        assert got == [2.0, 20.0, 5.0]
        assert rate == pytest.approx(2 * 10 / 20e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.replica_rate(1, 5, 10.0) == pytest.approx(500.0)
