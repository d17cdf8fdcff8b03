"""Database-sharded query: shard ranges and the exchange step, with 2 gloo ranks
on CPU (the device merge and the replicated S-IF are covered on the GPU in
tests/test_gpu_sharded.py)."""
import os
import socket

import numpy as np

from paper_1604_01879_gb300.sharded import shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _ref_merge(ids, sc, k):
    """Reference merge of candidate rows by (score desc, id asc) (test-side)."""
    out = []
    for bi, bs in zip(ids, sc):
        ok = bi >= 0
        bi, bs = bi[ok].astype(np.int64), bs[ok].astype(np.float64)
        out.append(bi[np.lexsort((bi, -bs))[:k]].tolist())
    return out


def test_shard_ranges_cover_the_database():
    for n, w in [(10, 3), (12000, 8), (7, 8)]:
        seen = []
        for r in range(w):
            b, m = shard_range(n, r, w)
            seen.extend(range(b, b + m))
        assert seen == list(range(n))


def _worker(rank, world, port, S, R, out):
    import torch
    import torch.distributed as dist
    from paper_1604_01879_gb300.sharded import exchange_topk, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        base, n = shard_range(S.shape[1], rank, world)
        loc = S[:, base:base + n]
        top = np.stack([np.lexsort((np.arange(n), -row))[:R] for row in loc])
        ids = torch.from_numpy(top.astype(np.int32))
        ids[:, -1] = -1  # an empty entry stays empty
        sc = torch.from_numpy(np.take_along_axis(loc, top, axis=1).astype(np.float32))
        gi, gs = exchange_topk(ids, sc, base)
        out[rank] = (gi.numpy().tolist(), gs.numpy().tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_global_candidates():
    """Each rank's local top-R, with its shard's base added, all-gathered rank-major:
    every rank holds the same [B, 2R] candidates, and their merge is the unsharded ranking."""
    import torch.multiprocessing as mp
    g = np.random.default_rng(1)
    S = np.round(g.random((4, 501)), 2).astype(np.float32)  # coarse values: ties across shards
    k, R, world = 25, 40, 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), S, R, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == out[1]
    ids, sc = np.asarray(out[0][0]), np.asarray(out[0][1])
    assert ids.shape == (4, world * R)
    assert (ids[:, R - 1] == -1).all() and (ids[:, 2 * R - 1] == -1).all()
    b1, _ = shard_range(S.shape[1], 1, world)
    assert (ids[:, R:2 * R - 1] >= b1).all() and (ids[:, :R - 1] < b1).all()
    merged = _ref_merge(ids, sc, k)
    for b in range(S.shape[0]):
        assert merged[b] == np.lexsort((np.arange(S.shape[1]), -S[b].astype(np.float64)))[:k].tolist()
