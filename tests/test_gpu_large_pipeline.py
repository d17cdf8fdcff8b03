"""The 200,000-shape pipeline at reduced size: counter-generated views drawn on the
device, streamed three-pass build, FP8 E4M3 store with per-view scales, query-side
MA = 2, FP32 rescore and S-IF re-rank, against the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import CONFIGS, config_views, config_codebook
from tests.parity import assert_topk, recall

pytestmark = pytest.mark.gpu

CFG = dataclasses.replace(CONFIGS["db200000x64_d4096_k4096_fp8"], name="counter_small", n_shapes=1200, dim=256,
                          n_classes=24, n_codewords=128, n_queries=12, kmeans_shapes=64, rescore_r=300, sif_k1=20)


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
