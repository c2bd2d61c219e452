"""Multi-replica host logic with two gloo ranks on CPU: max-over-ranks timing, summed work,
disjoint per-rank sources and the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    from paper_1312_3018_gb300 import replicas
    w, r, _ = replicas.init("gloo")
    assert (w, r) == (world, rank)
    replicas.barrier()
    slowest = replicas.max_over_ranks(10.0 * (rank + 1))      # ms
    units = replicas.sum_over_ranks(1000.0 * (rank + 1))
    mine = replicas.rank_slice(list(range(11)), rank, world)
    out[rank] = (slowest, units, mine, replicas.aggregate_rate(units, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of a threaded test process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] == out[1][1] == 3000.0
    a, b = out[0][2], out[1][2]
    assert not set(a) & set(b) and sorted(a + b) == list(range(11))
    assert out[0][3] == pytest.approx(3000.0 / 0.020)


def test_single_rank_is_identity(monkeypatch):
    from paper_1312_3018_gb300 import replicas
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.init("gloo") == (1, 0, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.sum_over_ranks(2.0) == 2.0
    assert replicas.rank_slice([1, 2, 3], 0, 1) == [1, 2, 3]

