"""Multi-rank helpers on CPU with gloo, world size 2: the query path shards
by queries with no exchange, so the only collectives are the barrier and the
max-over-ranks reduction of the timed region."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2607_16946_b300 import dist
    r, w, lr = dist.init(backend="gloo")
    assert (r, w, lr) == (rank, world, rank)
    dist.barrier()
    m = dist.max_over_ranks(1.5 + rank)
    b, e = dist.shard(1001, r, w)
    dist.finalize()
    q.put((rank, m, b, e))


def test_gloo_world_size_two():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [m for _, m, _, _ in res] == [2.5, 2.5]            # every rank sees the slowest time
    assert [(b, e) for _, _, b, e in res] == [(0, 501), (501, 1001)]


def test_shard_covers_everything():
    from paper_2607_16946_b300 import dist
    for total in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            spans = [dist.shard(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
