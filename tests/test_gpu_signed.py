"""Signed features on the GPU: Eq. 4 taken literally (a negative per-view maximum
counts only when every view of the shape shares a codeword with the query view),
on every scan path -- CUDA-core FP32 store, tensor-core BF16 and E4M3 scans,
the fused BF16 scan + FP32 rescore and the E4M3 store's FP32 rescore -- with
query- and database-side multiple assignment; K = 1 reduces Eq. 4 to Eq. 3
with negative scores; S-IF memberships of negative scores are 0."""
import numpy as np
import pytest

from oracle import gift_oracle as O
from tests.parity import ATOL, FIX, RTOL, ErrorBand, assert_topk, close, reference_memberships, sif_rows, sif_sets
from tests.signed_case import SIGNED, signed_case

pytestmark = pytest.mark.gpu


def _index(gift, X, cb, K, **kw):
    import torch
    N, Nv, _ = X.shape
    return gift.Index(torch.from_numpy(X).cuda(), torch.from_numpy(cb).cuda(), N, Nv, K, **kw)


def _full_rows(ix, Q, qoff, N, mode="fif"):
    import torch
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode=mode, topk=N)
    return ids.cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("ma,db_ma", [(1, 1), (2, 1), (1, 2), (3, 1)])
def test_signed_fif_full_rows_fp32_store(gpu_lib, ma, db_ma):
    X, cb, Q, qoff, dbc, qc = signed_case(ma=ma, db_ma=db_ma)
    N, K = SIGNED["N"], SIGNED["K"]
    ix = _index(gpu_lib, X, cb, K, storage="f32", query_ma=ma, db_ma=db_ma, keep_exact=ma == K)
    ids, sc = _full_rows(ix, Q, qoff, N)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    assert (ref < 0).any()
    for b in range(len(qoff) - 1):
        assert sorted(ids[b].tolist()) == list(range(N))
        assert close(sc[b], ref[b, ids[b]]).all(), b
        assert_topk(ids[b], sc[b], ref[b], N)
    if ma == K:  # every codeword: Eq. 4 is Eq. 3
        ref_e = O.exact_scores(Q, qoff, X)
        ide, sce = _full_rows(ix, Q, qoff, N, mode="exact")
        for b in range(len(qoff) - 1):
            assert close(sc[b], ref_e[b, ids[b]]).all()
            assert_topk(ide[b], sce[b], ref_e[b], N)
    ix.close()


@pytest.mark.parametrize("storage,ma", [("bf16", 1), ("bf16", 2), ("fp8", 1), ("fp8", 2)])
def test_signed_reduced_precision_store_with_fp32_rescore(gpu_lib, storage, ma):
    """Every shape rescored (R = N): the fused BF16 pass or the E4M3 store's rescore gives
    FP32-level scores of Eq. 4, negative terms included."""
    X, cb, Q, qoff, dbc, qc = signed_case(ma=ma)
    N, K = SIGNED["N"], SIGNED["K"]
    ix = _index(gpu_lib, X, cb, K, storage=storage, query_ma=ma, rescore_r=N, keep_exact=False)
    ids, sc = _full_rows(ix, Q, qoff, N)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(len(qoff) - 1):
        assert sorted(ids[b].tolist()) == list(range(N))
        assert close(sc[b], ref[b, ids[b]]).all(), b
        assert_topk(ids[b], sc[b], ref[b], N)
    ix.close()


@pytest.mark.parametrize("storage,tol", [("bf16", 3e-3), ("fp8", 6e-2)])
def test_signed_reduced_precision_store_without_rescore(gpu_lib, storage, tol):
    X, cb, Q, qoff, dbc, qc = signed_case(ma=2)
    N, K = SIGNED["N"], SIGNED["K"]
    ix = _index(gpu_lib, X, cb, K, storage=storage, query_ma=2, keep_exact=False)
    ids, sc = _full_rows(ix, Q, qoff, N)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(len(qoff) - 1):
        assert sorted(ids[b].tolist()) == list(range(N))
        assert np.abs(sc[b] - ref[b, ids[b]]).max() < tol
    ix.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_signed_one_codeword_fif_equals_exact(gpu_lib, storage):
    """K = 1: every view is matched, so Eq. 4 is Eq. 3 with its negative maxima."""
    X, cb, Q, qoff, dbc, qc = signed_case(K=1, N=120)
    N = 120
    ix = _index(gpu_lib, X, cb, 1, storage=storage, rescore_r=0 if storage == "f32" else N,
                keep_exact=storage == "f32")
    ids, sc = _full_rows(ix, Q, qoff, N)
    ref = O.exact_scores(Q, qoff, X)
    assert (ref < 0).any()
    for b in range(len(qoff) - 1):
        assert close(sc[b], ref[b, ids[b]]).all(), b
        assert_topk(ids[b], sc[b], ref[b], N)
    ix.close()


def test_signed_rerank_memberships_and_sprime(gpu_lib):
    """S-IF of a signed database (K = 1, two views per shape, k1 = 120 of 150 shapes, so
    many neighbours score below 0): such a neighbour has membership 0, memberships follow
    the oracle, and S' of the re-ranked shapes stays within the bound propagated from the
    memberships' FP32 error (tests/parity.py)."""
    import torch
    X, cb, Q, qoff, dbc, qc = signed_case(K=1, N=150, Nv=2, qviews=(2,))
    N, Nv, D = X.shape
    k1 = 120
    ix = _index(gpu_lib, X, cb, 1, storage="f32", sif_k1=k1, keep_exact=False)
    rows = X.reshape(-1, D)
    S_db = O.fif_scores(rows, np.arange(0, N * Nv + 1, Nv), O.quantize(rows, cb, 1), X, dbc)
    off, sids, mem, card = ix.export_sif()
    got, sets = sif_rows(off, sids, mem, N), sif_sets(off, sids, N)
    F_db = np.stack([reference_memberships(S_db[p], np.nonzero(sets[p])[0], k1) for p in range(N)])
    neg = sets & (S_db < -1e-4)
    assert neg.sum() >= 30  # neighbours with negative scores ...
    assert (got[neg] == 0).all()  # ... have membership 0
    assert close(got, F_db, RTOL, FIX / 2 + ATOL).all()
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=N)
    rid, rsp = ix.rerank(ids, sc, k1=k1, topk=10)
    ids, sc, rid, rsp = (t.cpu().numpy() for t in (ids, sc, rid, rsp))
    S_q = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(len(qoff) - 1):
        Fq = reference_memberships(S_q[b], ids[b, :k1], k1)
        gq = np.zeros(N)
        gq[ids[b, :k1]] = np.maximum(sc[b, :k1], 0.0)
        band = ErrorBand().add(got, F_db, floor=1e-3).add(gq, Fq, floor=1e-3)
        rtol, atol = band.sprime_tolerance(k1, Fq.sum())
        ref = np.array([O.contextual(Fq, F_db[p]) for p in range(N)])
        assert_topk(rid[b], rsp[b], ref, 10, rtol=rtol, atol=atol)
    ix.close()
