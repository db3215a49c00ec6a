"""Multi-process replica sharding on CPU (gloo, world size 2).

Replicas never interact, so running the replica blocks of one instance on two
ranks must give exactly the per-replica results of one process running all of
them, and the gathered best must be the single-process best.  The per-rank work
is the oracle (no GPU here); the sharding and the exchange are the code under test.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2412_09285_b300.sharding import best_over_ranks, shard_fields, shard_replicas


def test_shard_replicas_partitions_the_range():
    for total, world in [(32, 1), (64, 2), (96, 2), (1024, 8), (160, 3)]:
        seen = []
        for r in range(world):
            off, cnt = shard_replicas(total, world, r)
            assert off % 32 == 0 and cnt % 32 == 0 and cnt > 0
            seen += list(range(off, off + cnt))
        assert seen == list(range(total))
    with pytest.raises(ValueError):
        shard_replicas(48, 1, 0)
    with pytest.raises(ValueError):
        shard_replicas(32, 2, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle as O
    from paper_2412_09285_b300 import instances as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = I.er_gnp(120, 0.08, seed=5, weights="pm1")
    W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    h0 = I.initial_fields(g.n, 96, seed=6)
    mine = shard_fields(h0, world, rank).astype(np.float64)
    h, _ = O.anneal(("maxcut", W), mine, 200, mode="paper")
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, O.maxcut_states(h))
    r = O.best_replica(-cut)
    e, rep, owner = best_over_ranks(float(-cut[r]), r, rank, world)
    off, _ = shard_replicas(96, world, owner)
    out[rank] = (e, off + rep, [int(x) for x in cut])
    dist.destroy_process_group()


def test_two_rank_sharding_matches_single_process():
    import oracle as O
    from paper_2412_09285_b300 import instances as I
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    g = I.er_gnp(120, 0.08, seed=5, weights="pm1")
    W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    h0 = I.initial_fields(g.n, 96, seed=6).astype(np.float64)
    h, _ = O.anneal(("maxcut", W), h0, 200, mode="paper")
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, O.maxcut_states(h))
    # per-replica results are identical when split across ranks
    assert res[0][2] + res[1][2] == [int(x) for x in cut]
    best = O.best_replica(-cut)
    for r in range(world):
        assert res[r][0] == float(-cut[best]) and res[r][1] == best
