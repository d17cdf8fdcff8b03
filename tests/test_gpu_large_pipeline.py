"""The 200,000-shape pipeline at reduced size: counter-generated views drawn on the
device, streamed three-pass build, FP8 E4M3 store with per-view scales, query-side
MA = 2, FP32 rescore and S-IF re-rank, against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import CONFIGS, config_views, config_codebook
from tests.parity import ErrorBand, assert_topk, recall, reference_memberships, sif_rows, sif_sets

pytestmark = pytest.mark.gpu

CFG = dataclasses.replace(CONFIGS["db200000x64_d4096_k4096_fp8"], name="counter_small", n_shapes=1200, dim=256,
                          n_classes=24, n_codewords=128, n_queries=12, kmeans_shapes=64, rescore_r=300, sif_k1=20)
# small enough for the oracle to match every database shape as a query (its S-IF)
CFG_RR = dataclasses.replace(CFG, name="counter_rerank", n_shapes=360, n_views=32, n_classes=12, n_codewords=48,
                             n_queries=8, kmeans_shapes=48, rescore_r=120, sif_k1=12, topk=40)


def test_counter_views_identical_on_device(gpu_lib):
    import torch
    a = config_views(CFG, 37, 5)
    b = config_views(CFG, 37, 5, device="cuda").cpu().numpy()
    assert np.array_equal(a, b)


def test_streamed_fp8_ma2_pipeline_matches_oracle(gpu_lib):
    import torch
    cb = config_codebook(CFG)
    N, Nv, D, K = CFG.n_shapes, CFG.n_views, CFG.dim, CFG.n_codewords
    ix = gpu_lib.Index.streamed(lambda f, n: config_views(CFG, f, n, device="cuda"), torch.from_numpy(cb).cuda(),
                                N, Nv, K, chunk_shapes=250, storage="fp8", query_ma=CFG.query_ma,
                                sif_k1=CFG.sif_k1, rescore_r=CFG.rescore_r)
    X = config_views(CFG, 0, N)
    Q = config_views(CFG, 0, CFG.n_queries, query=True).reshape(-1, D)
    qoff = np.arange(CFG.n_queries + 1) * Nv
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=CFG.topk)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    dbc = O.quantize(X.reshape(-1, D), cb, 1).reshape(N, Nv)
    ref = O.fif_scores(Q, qoff, O.quantize(Q, cb, CFG.query_ma), X, dbc)
    rec = []
    for b in range(CFG.n_queries):
        assert_topk(ids[b], sc[b], ref[b], CFG.topk)  # FP32-rescored scores, ids at separated ranks
        rec.append(recall(ids[b], ref[b], CFG.topk))
    assert min(rec) >= 0.99
    rid, rsp = ix.rerank(torch.from_numpy(ids).cuda(), torch.from_numpy(sc).cuda(), k1=CFG.sif_k1, topk=10)
    assert rid.shape == (CFG.n_queries, 10) and torch.all(rsp[:, :-1] >= rsp[:, 1:])
    ix.close()


def test_streamed_fp8_ma2_rerank_matches_oracle(gpu_lib):
    """The same pipeline's S-IF re-rank against the oracle's own S-IF: the oracle matches
    every database shape as a query (Eq. 4, MA = 2) for its neighbour sets and memberships;
    re-ranked ids identical at separated ranks, S' within the bound propagated from the
    memberships' FP32 error (tests/parity.py)."""
    import torch
    c = CFG_RR
    cb = config_codebook(c)
    N, Nv, D, K, k1 = c.n_shapes, c.n_views, c.dim, c.n_codewords, c.sif_k1
    ix = gpu_lib.Index.streamed(lambda f, n: config_views(c, f, n, device="cuda"), torch.from_numpy(cb).cuda(),
                                N, Nv, K, chunk_shapes=100, storage="fp8", query_ma=c.query_ma, sif_k1=k1,
                                rescore_r=c.rescore_r)
    X = config_views(c, 0, N)
    rows = X.reshape(-1, D)
    dbc = O.quantize(rows, cb, 1).reshape(N, Nv)
    S_db = O.fif_scores(rows, np.arange(N + 1) * Nv, O.quantize(rows, cb, c.query_ma), X, dbc)
    off, sids, mem, _ = ix.export_sif()
    got, sets = sif_rows(off, sids, mem, N), sif_sets(off, sids, N)
    F_db = np.stack([reference_memberships(S_db[p], np.nonzero(sets[p])[0], k1) for p in range(N)])
    Q = config_views(c, 0, c.n_queries, query=True).reshape(-1, D)
    qoff = np.arange(c.n_queries + 1) * Nv
    S_q = O.fif_scores(Q, qoff, O.quantize(Q, cb, c.query_ma), X, dbc)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=c.topk)
    rid, rsp = ix.rerank(ids, sc, k1=k1, topk=10)
    ids, sc, rid, rsp = (t.cpu().numpy() for t in (ids, sc, rid, rsp))
    for b in range(c.n_queries):
        Fq = reference_memberships(S_q[b], ids[b, :k1], k1)
        gq = np.zeros(N)
        gq[ids[b, :k1]] = np.maximum(sc[b, :k1], 0.0)
        band = ErrorBand().add(got, F_db).add(gq, Fq)
        rtol, atol = band.sprime_tolerance(k1, Fq.sum())
        assert rtol <= 1e-5, (band.lo, band.hi)
        ref = np.array([O.contextual(Fq, F_db[p]) for p in range(N)])
        assert_topk(rid[b], rsp[b], ref, 10, rtol=rtol, atol=atol)
    ix.close()
