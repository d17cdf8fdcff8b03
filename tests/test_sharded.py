"""Database-sharded query: the exchange and merge, with 2 gloo ranks on CPU."""
import os
import socket

import numpy as np
import pytest

from paper_1604_01879_gb300.sharded import merge_topk, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_merge_equals_global_ranking_with_ties():
    g = np.random.default_rng(0)
    B, N, k = 5, 300, 20
    S = np.round(g.random((B, N)), 2)  # coarse values: many ties across shards
    shards = [(0, 110), (110, 90), (200, 100)]
    ids_l, sc_l = [], []
    for base, n in shards:
        loc = S[:, base:base + n]
        top = np.stack([np.lexsort((np.arange(n), -row))[:k] for row in loc])
        ids_l.append(top + base)
        sc_l.append(np.take_along_axis(loc, top, axis=1))
    mi, ms = merge_topk(ids_l, sc_l, k)
    for b in range(B):
        ref = np.lexsort((np.arange(N), -S[b]))[:k]
        assert mi[b].tolist() == ref.tolist()
        assert np.allclose(ms[b], S[b, ref])


def test_merge_pads_when_shards_are_short():
    mi, ms = merge_topk([np.array([[3, -1]])], [np.array([[0.5, -np.inf]])], 4)
    assert mi.tolist() == [[3, -1, -1, -1]] and np.isneginf(ms[0, 1:]).all()


def test_shard_ranges_cover_the_database():
    for n, w in [(10, 3), (12000, 8), (7, 8)]:
        seen = []
        for r in range(w):
            b, m = shard_range(n, r, w)
            seen.extend(range(b, b + m))
        assert seen == list(range(n))


def _worker(rank, world, port, S, k, R, out):
    import torch
    import torch.distributed as dist
    from paper_1604_01879_gb300.sharded import sharded_topk, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        base, n = shard_range(S.shape[1], rank, world)
        loc = S[:, base:base + n]
        top = np.stack([np.lexsort((np.arange(n), -row))[:R] for row in loc])
        ids = torch.from_numpy(top.astype(np.int32))
        sc = torch.from_numpy(np.take_along_axis(loc, top, axis=1).astype(np.float32))
        gi, gs = sharded_topk(ids, sc, base, k)
        out[rank] = (gi.tolist(), gs.tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_with_unsharded_ranking():
    import torch.multiprocessing as mp
    g = np.random.default_rng(1)
    S = g.random((4, 501)).astype(np.float32)
    k, R, world = 25, 40, 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), S, k, R, out), nprocs=world, join=True,
                       start_method="spawn")
    for b in range(S.shape[0]):
        ref = np.lexsort((np.arange(S.shape[1]), -S[b].astype(np.float64)))[:k]
        for r in range(world):
            assert out[r][0][b] == ref.tolist()
    assert out[0] == out[1]
