"""Database-sharded query across ranks (one GPU per rank).

Each rank holds the F-IF of its own contiguous range of database shapes
[base, base + n_local) and answers a query batch on that shard; one
all-gather of every rank's top-R (global shape id, score) pairs per query
follows, and every rank merges them into the global top-k in the ranking
order (score desc, id asc). Eq. 4 scores of a shape depend only on that
shape's views, so the merged list equals the top-k of an unsharded index.

The exchange is the only collective; it moves B * R * 8 bytes per rank.
"""
from __future__ import annotations

import numpy as np


def merge_topk(ids_list, scores_list, k: int):
    """Merge per-shard ranked lists (global ids) into the top-k by (score desc, id asc).

    ids_list / scores_list: sequences of arrays [B, R_s]; invalid entries have id < 0.
    Returns (ids int64 [B, k], scores float64 [B, k]); missing entries are -1 / -inf.
    """
    ids = np.concatenate([np.asarray(a) for a in ids_list], axis=1).astype(np.int64)
    sc = np.concatenate([np.asarray(a) for a in scores_list], axis=1).astype(np.float64)
    B = ids.shape[0]
    out_i = np.full((B, k), -1, np.int64)
    out_s = np.full((B, k), -np.inf)
    for b in range(B):
        ok = ids[b] >= 0
        bi, bs = ids[b][ok], sc[b][ok]
        order = np.lexsort((bi, -bs))[:k]
        out_i[b, :len(order)] = bi[order]
        out_s[b, :len(order)] = bs[order]
    return out_i, out_s


def sharded_topk(local_ids, local_scores, base: int, k: int, group=None):
    """All-gather every rank's local top-R (ids local to its shard) and merge.

    local_ids int [B, R], local_scores float [B, R] (CPU or CUDA tensors);
    base is the first global shape id of this rank's shard. Returns the
    global top-k (ids, scores) as numpy arrays on every rank.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gid = torch.where(local_ids >= 0, local_ids.to(torch.int64) + int(base), torch.full_like(local_ids, -1,
                                                                                             dtype=torch.int64))
    sc = local_scores.to(torch.float64)
    g_ids = [torch.empty_like(gid) for _ in range(world)]
    g_sc = [torch.empty_like(sc) for _ in range(world)]
    dist.all_gather(g_ids, gid, group=group)
    dist.all_gather(g_sc, sc, group=group)
    return merge_topk([t.cpu().numpy() for t in g_ids], [t.cpu().numpy() for t in g_sc], k)


def shard_range(n_shapes: int, rank: int, world: int):
    """Contiguous shard [base, base + n) of rank among world ranks."""
    per = (n_shapes + world - 1) // world
    base = min(n_shapes, rank * per)
    return base, min(n_shapes, base + per) - base


class ShardedIndex:
    """A rank's shard of the database behind the same query call as Index."""

    def __init__(self, db_feats_shard, codebook, base: int, n_total: int, views_per_shape: int, n_codewords: int,
                 **index_kw):
        from . import Index
        self.base = int(base)
        self.n_total = int(n_total)
        self.n_local = int(db_feats_shard.shape[0]) // views_per_shape if db_feats_shard.ndim == 2 else \
            int(db_feats_shard.shape[0])
        self.local = Index(db_feats_shard, codebook, self.n_local, views_per_shape, n_codewords, **index_kw)

    def query(self, q_feats, q_offsets, topk: int = 10, depth: int | None = None, group=None):
        """Global top-k of a query batch: local F-IF top-`depth` on this shard, all-gather, merge."""
        depth = topk if depth is None else depth
        ids, sc = self.local.query(q_feats, q_offsets, mode="fif", topk=depth)
        return sharded_topk(ids, sc, self.base, topk, group=group)

    def close(self):
        self.local.close()
