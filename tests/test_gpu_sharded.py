"""Database-sharded query on one GPU: the device merge of shard lists
(gift_merge_topk) and the replicated S-IF of a sharded database
(gift_sif_from_neighbours) against an unsharded index. The all-gather of the
multi-rank path is emulated by concatenating the shards' lists in rank order,
which is what exchange_topk returns (tested with gloo ranks on CPU)."""
import numpy as np
import pytest

from paper_1604_01879_gb300.sharded import shard_range
from synth import kmeans_codebook, query_views, shape_views

pytestmark = pytest.mark.gpu


def _ref_merge(ids, sc, k):
    out_i, out_s = [], []
    for bi, bs in zip(ids, sc):
        ok = bi >= 0
        bi, bs = bi[ok].astype(np.int64), bs[ok].astype(np.float64)
        o = np.lexsort((bi, -bs))[:k]
        pad = k - len(o)
        out_i.append(bi[o].tolist() + [-1] * pad)
        out_s.append(bs[o].tolist() + [-np.inf] * pad)
    return np.asarray(out_i), np.asarray(out_s)


@pytest.mark.parametrize("B,n,k", [(5, 60, 20), (3, 3000, 100), (2, 7, 10)])
def test_device_merge_equals_reference_with_ties_and_short_rows(gpu_lib, B, n, k):
    import torch
    g = np.random.default_rng(n)
    sc = np.round(g.random((B, n)), 2).astype(np.float32)  # many equal scores: ties go to the lower id
    ids = np.stack([g.permutation(10 * n)[:n] for _ in range(B)]).astype(np.int32)
    ids[:, ::7] = -1  # empty entries
    oi, os_ = gpu_lib.merge_topk(torch.from_numpy(ids).cuda(), torch.from_numpy(sc).cuda(), k)
    ri, rs = _ref_merge(ids, sc, k)
    assert np.array_equal(oi.cpu().numpy(), ri)
    assert np.array_equal(os_.cpu().numpy(), rs.astype(np.float32))
    # host buffers through the same call
    hi, hs = np.empty((B, k), np.int32), np.empty((B, k), np.float32)
    gpu_lib.merge_topk(ids, sc, k, out=(hi, hs))
    torch.cuda.synchronize()
    assert np.array_equal(hi, ri)


def test_sharded_query_and_rerank_equal_the_unsharded_index(gpu_lib):
    """Two shards: merged top-k of the shards' lists = the unsharded top-k; the S-IF built
    from the merged neighbour rows of every database shape, installed on each shard, gives
    the unsharded index's S-IF and re-ranking, bit for bit."""
    import torch
    N, Nv, D, C, K, k1 = 150, 16, 64, 5, 10, 8
    X = shape_views(0, N, Nv, D, C, 1111, 4111)
    cb = kmeans_codebook(X.reshape(-1, D), K, 3111, 8)
    Q, qoff, _ = query_views(7, (16, 9), D, C, 2111, 4111, max_views=16)
    dev_cb = torch.from_numpy(cb).cuda()
    full = gpu_lib.Index(torch.from_numpy(X).cuda(), dev_cb, N, Nv, K, storage="f32", sif_k1=k1, keep_exact=False)
    shards = []
    for r in range(2):
        base, n = shard_range(N, r, 2)
        shards.append((base, gpu_lib.Index(torch.from_numpy(np.ascontiguousarray(X[base:base + n])).cuda(), dev_cb,
                                           n, Nv, K, storage="f32", keep_exact=False)))

    def sharded_query(q, off, k):
        parts = [ix.query(q, off, mode="fif", topk=k) for _, ix in shards]
        ids = torch.cat([torch.where(i >= 0, i + base, torch.full_like(i, -1)) for (base, _), (i, _) in
                         zip(shards, parts)], dim=1).contiguous()
        sc = torch.cat([s for _, s in parts], dim=1).contiguous()
        return gpu_lib.merge_topk(ids, sc, k)

    qd = torch.from_numpy(Q).cuda()
    fi, fs = full.query(qd, qoff, mode="fif", topk=40)
    si, ss = sharded_query(qd, qoff, 40)
    assert torch.equal(fi, si) and torch.equal(fs, ss)
    # replicated S-IF from the merged neighbour rows of every database shape
    rows = torch.from_numpy(X.reshape(-1, D)).cuda()
    off = np.arange(N + 1, dtype=np.int32) * Nv
    ni, ns = sharded_query(rows, off, k1)
    for _, ix in shards:
        ix.set_sif(ni, ns, N, k1)
        for a, b in zip(full.export_sif(), ix.export_sif()):
            assert np.array_equal(a, b)
    fr = full.rerank(fi, fs, k1=k1, topk=10)
    for _, ix in shards:
        sr = ix.rerank(si, ss, k1=k1, topk=10)
        assert torch.equal(fr[0], sr[0]) and torch.equal(fr[1], sr[1])
    # a shard index accepts one S-IF only
    with pytest.raises(gpu_lib.GiftError):
        shards[0][1].set_sif(ni, ns, N, k1)
    for _, ix in shards:
        ix.close()
    full.close()
