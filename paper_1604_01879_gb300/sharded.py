"""Database-sharded query across ranks (one GPU per rank).

Each rank holds the F-IF of its own contiguous range of database shapes
[base, base + n_local) and answers a query batch on that shard; one
all-gather of every rank's top-R (global shape id, score) pairs per query
follows, and the library merges them on the device into the global top-k in
the ranking order (score desc, id asc) (gift_merge_topk). Eq. 4 scores of a
shape depend only on that shape's views, so the merged list equals the top-k
of an unsharded index.

The second inverted file (Sec. 2.4) is replicated: every database shape is
queried against every shard in the same way (an off-line step), the merged
top-k1 rows give its activation, and each rank installs the S-IF of the whole
database from them (gift_sif_from_neighbours). Re-ranking then needs no
exchange: every rank re-ranks the merged candidates over the replicated S-IF.

The exchange is the only collective; it moves B * R * 8 bytes per rank per
query batch.
"""
from __future__ import annotations


def shard_range(n_shapes: int, rank: int, world: int):
    """Contiguous shard [base, base + n) of rank among world ranks."""
    per = (n_shapes + world - 1) // world
    base = min(n_shapes, rank * per)
    return base, min(n_shapes, base + per) - base


def exchange_topk(local_ids, local_scores, base: int, group=None):
    """All-gather every rank's local top-R (ids local to its shard, int32 [B, R];
    scores float32 [B, R]) as global candidates: (ids int32, scores float32)
    [B, world * R], rank-major; empty entries (id < 0) stay -1. The tensors stay on
    their device (NCCL for CUDA tensors, gloo for host tensors)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gid = torch.where(local_ids >= 0, local_ids + int(base), torch.full_like(local_ids, -1)).contiguous()
    sc = local_scores.contiguous()
    g_ids = [torch.empty_like(gid) for _ in range(world)]
    g_sc = [torch.empty_like(sc) for _ in range(world)]
    dist.all_gather(g_ids, gid, group=group)
    dist.all_gather(g_sc, sc, group=group)
    return torch.cat(g_ids, dim=1), torch.cat(g_sc, dim=1)


def sharded_topk(local_ids, local_scores, base: int, k: int, group=None, stream=None):
    """Global top-k of a batch from every rank's local top-R (CUDA tensors): the
    exchange, then the device merge (gift_merge_topk). Same result on every rank."""
    from . import merge_topk
    ids, sc = exchange_topk(local_ids, local_scores, base, group)
    return merge_topk(ids, sc, k, stream=stream)


class ShardedIndex:
    """A rank's shard of the database behind the same calls as Index."""

    def __init__(self, db_feats_shard, codebook, base: int, n_total: int, views_per_shape: int, n_codewords: int,
                 **index_kw):
        from . import Index
        if index_kw.get("sif_k1"):
            raise ValueError("a shard's S-IF covers the whole database: build it with build_sif")
        self.base = int(base)
        self.n_total = int(n_total)
        self.views_per_shape = int(views_per_shape)
        self.n_local = int(db_feats_shard.shape[0]) // views_per_shape if db_feats_shard.ndim == 2 else \
            int(db_feats_shard.shape[0])
        self.local = Index(db_feats_shard, codebook, self.n_local, views_per_shape, n_codewords, **index_kw)

    def query(self, q_feats, q_offsets, topk: int = 10, depth: int | None = None, group=None, stream=None):
        """Global top-k of a query batch: local F-IF top-`depth` on this shard, all-gather, device merge."""
        depth = topk if depth is None else depth
        ids, sc = self.local.query(q_feats, q_offsets, mode="fif", topk=depth, stream=stream)
        return sharded_topk(ids, sc, self.base, topk, group=group, stream=stream)

    def build_sif(self, views_of, k1: int, chunk_shapes: int = 256, group=None, stream=None):
        """The S-IF of the whole database, replicated on this rank: every database shape
        (views_of(first, n) gives the float32 views [n, N_v, D] of global shapes
        [first, first + n), on every rank) is queried on this shard, the shards' top-k1
        are exchanged and merged, and the merged rows (N_k1 of each shape, itself
        included, with its scores) are installed as the S-IF (gift_sif_from_neighbours)."""
        import numpy as np
        import torch
        rows_i, rows_s = [], []
        nv = self.views_per_shape
        for first in range(0, self.n_total, chunk_shapes):
            n = min(chunk_shapes, self.n_total - first)
            x = views_of(first, n)
            x = x.reshape(n * nv, -1)
            off = np.arange(n + 1, dtype=np.int32) * nv
            ids, sc = self.query(x, off, topk=k1, group=group, stream=stream)
            rows_i.append(ids)
            rows_s.append(sc)
        ids = torch.cat(rows_i).contiguous()
        sc = torch.cat(rows_s).contiguous()
        self.local.set_sif(ids, sc, self.n_total, k1, stream=stream)

    def rerank(self, cand_ids, cand_scores, k1: int, topk: int = 10, stream=None):
        """S-IF re-ranking of merged (global) candidates over the replicated S-IF; no exchange."""
        return self.local.rerank(cand_ids, cand_scores, k1=k1, topk=topk, stream=stream)

    def close(self):
        self.local.close()
