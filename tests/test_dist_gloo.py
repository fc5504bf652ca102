"""Interval sharding and max-over-ranks timing with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1709_08681_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = D.rank_info()
    ms = D.max_over_ranks(10.0 + r)
    b, e = D.shard_intervals(7, ws, r)
    dist.barrier()
    q.put((r, ms, b, e, D.rank_seed(5, r)))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [11.0, 11.0]          # max over ranks on both
    assert [(o[2], o[3]) for o in out] == [(0, 4), (4, 7)]
    assert out[0][4] != out[1][4]


def test_shards_cover_every_interval_once():
    for n in (0, 1, 5, 256):
        for ws in (1, 2, 3, 8):
            spans = [D.shard_intervals(n, ws, r) for r in range(ws)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[k][1] == spans[k + 1][0] for k in range(ws - 1))
            assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1
