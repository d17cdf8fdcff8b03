"""CUDA path vs the FP64 oracle, element by element, on seeded inputs.

Sizes span several scan tiles (64 entries x 64 slots), several GEMM tiles
(128 x 128) and ragged tails; edge cases: K = 1, MA up to 3, view counts that
differ per query, database smaller than k, host buffers.
"""
import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import CONFIGS, make_config_inputs, shape_views, query_views, kmeans_codebook
from tests.parity import (ATOL, FIX, RTOL, ErrorBand, assert_codes, assert_topk, close, code_margins, recall,
                          reference_memberships, sif_rows, sif_sets)

pytestmark = pytest.mark.gpu


def _case(N, Nv, D, C, K, nq, views, seed, ma=1):
    X = shape_views(0, N, Nv, D, C, 1000 + seed, 4000 + seed)
    cb = kmeans_codebook(X.reshape(-1, D), K, 3000 + seed, 8)
    Q, qoff, _ = query_views(nq, views, D, C, 2000 + seed, 4000 + seed, max_views=max(views))
    dbc = O.quantize(X.reshape(-1, D), cb, 1).reshape(N, Nv)
    qc = O.quantize(Q, cb, ma)
    return X, cb, Q, qoff, dbc, qc


def _index(gift, torch, X, cb, N, Nv, K, **kw):
    return gift.Index(torch.from_numpy(X).cuda(), torch.from_numpy(cb).cuda(), N, Nv, K, **kw)


@pytest.fixture(scope="module")
def c1(gpu_lib):
    import torch
    cfg = CONFIGS["db200x64_d128_k64"]
    d = make_config_inputs(cfg)
    X, cb, Q, qoff = d["db"], d["codebook"], d["q"], d["q_off"]
    N, Nv, D, K = cfg.n_shapes, cfg.n_views, cfg.dim, cfg.n_codewords
    dbc = O.quantize(X.reshape(-1, D), cb, 1).reshape(N, Nv)
    qc = O.quantize(Q, cb, 1)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="f32", sif_k1=cfg.sif_k1, keep_exact=True)
    yield dict(cfg=cfg, X=X, cb=cb, Q=Q, qoff=qoff, dbc=dbc, qc=qc, ix=ix)
    ix.close()


# ------------------------------------------------------------------ quantiser
@pytest.mark.parametrize("ma", [1, 2, 3])
def test_assign_matches_oracle(c1, ma):
    import torch
    Q, cb = c1["Q"], c1["cb"]
    got = c1["ix"].assign(torch.from_numpy(Q).cuda(), ma).cpu().numpy()
    ref = O.quantize(Q, cb, ma)
    n_bad, n_tied = assert_codes(got, ref, code_margins(Q, cb, ma))
    assert n_bad <= n_tied


def test_assign_database_rows_all_codewords(c1):
    import torch
    X, cb = c1["X"], c1["cb"]
    rows = X.reshape(-1, X.shape[2])
    got = c1["ix"].assign(torch.from_numpy(rows).cuda(), 1).cpu().numpy()
    assert_codes(got, O.quantize(rows, cb, 1), code_margins(rows, cb, 1))


# ------------------------------------------------------------------ F-IF structure
def test_posting_lists_identical(c1):
    codes, off, rows = c1["ix"].export_fif()
    N, Nv = c1["dbc"].shape
    assert_codes(codes.reshape(-1, 1), c1["dbc"].reshape(-1, 1),
                 code_margins(c1["X"].reshape(N * Nv, -1), c1["cb"], 1))
    lists = O.build_fif(c1["dbc"], c1["cb"].shape[0])  # the oracle's lists from the oracle's codes
    assert off[0] == 0 and off[-1] == N * Nv
    for k, l in enumerate(lists):
        assert off[k + 1] - off[k] == len(l)
        ref = (l[:, 0] * Nv + l[:, 1]) if len(l) else np.zeros(0, np.int64)
        assert np.array_equal(rows[off[k]:off[k + 1]], ref)
        # rows strictly ascending: the runs of equal shape are strictly ascending in shape
        assert np.all(np.diff(rows[off[k]:off[k + 1]]) > 0)


# ------------------------------------------------------------------ scores and top-k
def test_exact_query_small_config(c1):
    import torch
    ids, sc = c1["ix"].query(torch.from_numpy(c1["Q"]).cuda(), c1["qoff"], mode="exact", topk=10)
    ref = O.exact_scores(c1["Q"], c1["qoff"], c1["X"])
    for b in range(len(c1["qoff"]) - 1):
        assert_topk(ids[b].cpu().numpy(), sc[b].cpu().numpy(), ref[b], 10)


def test_fif_query_small_config(c1):
    import torch
    ids, sc = c1["ix"].query(torch.from_numpy(c1["Q"]).cuda(), c1["qoff"], mode="fif", topk=10)
    ref = O.fif_scores(c1["Q"], c1["qoff"], c1["qc"], c1["X"], c1["dbc"])
    for b in range(len(c1["qoff"]) - 1):
        assert_topk(ids[b].cpu().numpy(), sc[b].cpu().numpy(), ref[b], 10)


def test_fif_full_rows_small_config(c1):
    """topk = N: every shape's F-IF score, compared element by element."""
    import torch
    N = c1["cfg"].n_shapes
    ids, sc = c1["ix"].query(torch.from_numpy(c1["Q"]).cuda(), c1["qoff"], mode="fif", topk=N)
    ref = O.fif_scores(c1["Q"], c1["qoff"], c1["qc"], c1["X"], c1["dbc"])
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for b in range(ids.shape[0]):
        assert sorted(ids[b].tolist()) == list(range(N))
        assert close(sc[b], ref[b, ids[b]]).all()


@pytest.mark.parametrize("ma", [1, 2, 3])
def test_fif_ragged_multiple_assignment(gpu_lib, ma):
    """N, N_v, V_q not multiples of any tile; lists longer than a scan tile."""
    import torch
    N, Nv, D, C, K = 37, 20, 48, 4, 6
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 9, (5, 12, 20, 33), 31, ma)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="f32", query_ma=ma, keep_exact=True)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=N)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for b in range(len(qoff) - 1):
        assert close(sc[b], ref[b, ids[b]]).all(), b
        assert_topk(ids[b], sc[b], ref[b], N)
    ids_e, sc_e = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="exact", topk=N)
    ref_e = O.exact_scores(Q, qoff, X)
    for b in range(len(qoff) - 1):
        assert_topk(ids_e[b].cpu().numpy(), sc_e[b].cpu().numpy(), ref_e[b], N)
    ix.close()


def test_many_slots_per_list(gpu_lib):
    """K = 3 codewords: every list is long and is hit by many query views (slot chunks)."""
    import torch
    N, Nv, D, C, K = 300, 16, 32, 3, 3
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 40, (16, 7), 41)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="f32", keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=50)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(len(qoff) - 1):
        assert_topk(ids[b].cpu().numpy(), sc[b].cpu().numpy(), ref[b], 50)
    ix.close()


def test_one_codeword_fif_equals_exact(gpu_lib):
    """K = 1: Eq. 4 reduces to Eq. 3 on the GPU as in the oracle."""
    import torch
    N, Nv, D = 50, 24, 64
    X = shape_views(0, N, Nv, D, 5, 1051, 4051)
    cb = np.ones((1, D), np.float32)
    Q, qoff, _ = query_views(6, (24, 9), D, 5, 2051, 4051, max_views=24)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, 1, storage="f32", keep_exact=True)
    qd = torch.from_numpy(Q).cuda()
    ids_f, sc_f = ix.query(qd, qoff, mode="fif", topk=N)
    ids_e, sc_e = ix.query(qd, qoff, mode="exact", topk=N)
    ref = O.exact_scores(Q, qoff, X)
    for b in range(len(qoff) - 1):
        assert_topk(ids_f[b].cpu().numpy(), sc_f[b].cpu().numpy(), ref[b], N)
        assert_topk(ids_e[b].cpu().numpy(), sc_e[b].cpu().numpy(), ref[b], N)
    ix.close()


def test_self_match_ranks_first(c1):
    import torch
    X = c1["X"]
    N, Nv, D = X.shape
    pick = [0, 17, 199]
    Q = np.concatenate([X[p] for p in pick])
    qoff = np.arange(0, len(pick) * Nv + 1, Nv, dtype=np.int32)
    for mode in ("fif", "exact"):
        ids, sc = c1["ix"].query(torch.from_numpy(Q).cuda(), qoff, mode=mode, topk=3)
        assert ids[:, 0].cpu().tolist() == pick
        assert np.allclose(sc[:, 0].cpu().numpy(), 1.0, atol=2e-6)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_reduced_precision_store_with_fp32_rescore(gpu_lib, storage):
    """BF16 / FP8 store, top-R rescored in FP32: scores FP32-accurate."""
    import torch
    N, Nv, D, C, K = 160, 32, 128, 8, 24
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 12, (32,), 61)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage=storage, rescore_r=60, keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=20)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(len(qoff) - 1):
        assert_topk(ids[b].cpu().numpy(), sc[b].cpu().numpy(), ref[b], 20)
    ix.close()


@pytest.mark.parametrize("storage,tol", [("bf16", 3e-3), ("fp8", 6e-2)])
def test_reduced_precision_store_without_rescore(gpu_lib, storage, tol):
    import torch
    N, Nv, D, C, K = 120, 32, 128, 6, 16
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 8, (32,), 71)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage=storage, keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=N)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(len(qoff) - 1):
        i = ids[b].cpu().numpy()
        assert np.abs(sc[b].cpu().numpy() - ref[b, i]).max() < tol
    ix.close()


def test_fp8_lists_of_every_slot_class(gpu_lib):
    """E4M3 scan and FP32-level rescore with query MA = 2 where the touched lists hold from 16 to
    386 query slots: lists of up to 80 slots run with entries as the MMA rows (slot tiles of 16,
    32, 64, 80), larger ones with slots as the rows, in one or several slot tiles of 128."""
    import torch
    N, Nv, D, C, K = 96, 16, 128, 4, 12
    X, cb, _, _, dbc, _ = _case(N, Nv, D, C, K, 1, (16,), 151)
    picks = [c + C * i for c, n in enumerate((24, 12, 5, 1)) for i in range(n)]  # queries per class
    Q = np.concatenate([X[p] for p in picks])
    qoff = np.arange(len(picks) + 1, dtype=np.int32) * Nv
    qc = O.quantize(Q, cb, 2)
    M = np.bincount(qc.ravel(), minlength=K)
    M = M[M > 0]
    assert (M <= 16).any() and ((M > 16) & (M <= 32)).any() and ((M > 32) & (M <= 64)).any()
    assert ((M > 64) & (M <= 80)).any() and ((M > 80) & (M <= 128)).any() and (M > 256).any()
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    Qd = torch.from_numpy(Q).cuda()
    plain = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="fp8", query_ma=2, keep_exact=False)
    ids, sc = plain.query(Qd, qoff, mode="fif", topk=N)
    for b in range(len(picks)):
        i = ids[b].cpu().numpy()
        assert sorted(i.tolist()) == list(range(N))
        assert np.abs(sc[b].cpu().numpy() - ref[b, i]).max() < 6e-2
    plain.close()
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="fp8", query_ma=2, rescore_r=64, keep_exact=False)
    ids, sc = ix.query(Qd, qoff, mode="fif", topk=20)
    for b in range(len(picks)):
        assert_topk(ids[b].cpu().numpy(), sc[b].cpu().numpy(), ref[b], 20)
    ix.close()


def test_database_smaller_than_k(gpu_lib):
    import torch
    N, Nv, D, C, K = 5, 8, 16, 2, 3
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 2, (8,), 81)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="f32", keep_exact=True)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=8)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    assert (ids[:, N:] == -1).all() and np.isneginf(sc[:, N:]).all()
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    for b in range(2):
        assert_topk(ids[b, :N], sc[b, :N], ref[b], N)
    ix.close()


def test_host_buffers_match_device(c1):
    import torch
    Q = c1["Q"]
    ids_d, sc_d = c1["ix"].query(torch.from_numpy(Q).cuda(), c1["qoff"], mode="fif", topk=10)
    out = (np.empty((len(c1["qoff"]) - 1, 10), np.int32), np.empty((len(c1["qoff"]) - 1, 10), np.float32))
    qh = torch.from_numpy(Q).pin_memory()
    c1["ix"].query(qh, c1["qoff"], mode="fif", topk=10, out=out)
    torch.cuda.synchronize()
    assert np.array_equal(out[0], ids_d.cpu().numpy())
    assert np.array_equal(out[1], sc_d.cpu().numpy())


def test_invalid_arguments_rejected(c1):
    import torch
    import paper_1604_01879_gb300 as gift
    qd = torch.from_numpy(c1["Q"]).cuda()
    with pytest.raises(gift.GiftError):
        c1["ix"].query(qd, c1["qoff"], mode="fif", topk=2000)
    bad = np.array(c1["qoff"]).copy()
    bad[2] = bad[1]
    with pytest.raises(gift.GiftError):
        c1["ix"].query(qd, bad, mode="fif", topk=10)
    with pytest.raises(gift.GiftError):
        gift.Index(torch.zeros((4, 2, 20), device="cuda"), torch.zeros((3, 20), device="cuda"), 4, 2, 3)


# ------------------------------------------------------------------ S-IF
def _oracle_sif(X, dbc, cb, k1):
    N, Nv, D = X.shape
    rows = X.reshape(-1, D)
    S_db = O.fif_scores(rows, np.arange(0, N * Nv + 1, Nv), O.quantize(rows, cb, 1), X, dbc)
    return S_db, O.db_memberships(S_db, k1)


def test_sif_entries_match_oracle(c1):
    X, dbc, cb = c1["X"], c1["dbc"], c1["cb"]
    k1 = c1["cfg"].sif_k1
    N = X.shape[0]
    S_db, _ = _oracle_sif(X, dbc, cb, k1)
    off, ids, mem, card = c1["ix"].export_sif()
    assert off[-1] == N * k1
    got, sets = sif_rows(off, ids, mem, N), sif_sets(off, ids, N)
    for p in range(N):
        # N_k1(p) is a correct first-k1 set (unique away from near ties at the k1 boundary)
        F_ref = reference_memberships(S_db[p], np.nonzero(sets[p])[0], k1)
        srt = -np.sort(-S_db[p])
        if srt[k1 - 1] - srt[k1] > 2 * (RTOL * srt[k1 - 1] + ATOL):
            assert np.array_equal(np.nonzero(sets[p])[0], np.nonzero(O.membership(S_db[p], k1))[0]), p
        # memberships: FP32 scores (score tolerance) in fixed point (half a step)
        assert close(got[p], F_ref, RTOL, FIX / 2).all(), p
        assert abs(card[p] * FIX - F_ref.sum()) <= RTOL * F_ref.sum() + k1 * FIX / 2
    for i in range(N):
        assert np.all(np.diff(ids[off[i]:off[i + 1]]) > 0)  # p ascending


def test_rerank_matches_oracle(c1):
    """S' of Eq. 8 within the bound propagated from the memberships' FP32 error (tests/parity.py),
    re-ranked ids identical at separated ranks; the oracle's memberships are taken on the GPU's
    neighbour sets once those are checked to be correct first-k1 sets."""
    import torch
    X, dbc, cb, Q, qoff = c1["X"], c1["dbc"], c1["cb"], c1["Q"], c1["qoff"]
    k1 = c1["cfg"].sif_k1
    N = X.shape[0]
    S_db, _ = _oracle_sif(X, dbc, cb, k1)
    off, sids, mem, _ = c1["ix"].export_sif()
    got, sets = sif_rows(off, sids, mem, N), sif_sets(off, sids, N)
    F_db = np.stack([reference_memberships(S_db[p], np.nonzero(sets[p])[0], k1) for p in range(N)])
    S_q = O.fif_scores(Q, qoff, c1["qc"], X, dbc)
    ids, sc = c1["ix"].query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=30)
    rid, rsp = c1["ix"].rerank(ids, sc, k1=k1, topk=10)
    ids, sc, rid, rsp = (t.cpu().numpy() for t in (ids, sc, rid, rsp))
    for b in range(len(qoff) - 1):
        Fq = reference_memberships(S_q[b], ids[b, :k1], k1)
        gq = np.zeros(N)
        gq[ids[b, :k1]] = np.maximum(sc[b, :k1], 0.0)
        band = ErrorBand().add(got, F_db).add(gq, Fq)
        rtol, atol = band.sprime_tolerance(k1, Fq.sum())
        assert rtol <= 1e-5, (band.lo, band.hi)
        ref = np.array([O.contextual(Fq, F_db[p]) for p in range(N)])
        assert_topk(rid[b], rsp[b], ref, 10, rtol=rtol, atol=atol)


def test_rerank_whole_database_order(c1):
    """topk = N: every shape once, by S' (Eq. 8) desc, then the F-IF score S desc for candidates,
    then ascending id for the shapes neither the S-IF walk nor the candidate list reaches."""
    import torch
    Q, qoff = c1["Q"], c1["qoff"]
    k1, N = c1["cfg"].sif_k1, c1["X"].shape[0]
    ids, sc = c1["ix"].query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=30)
    rid, rsp = c1["ix"].rerank(ids, sc, k1=k1, topk=N)
    ids, sc, rid, rsp = (t.cpu().numpy() for t in (ids, sc, rid, rsp))
    for b in range(len(qoff) - 1):
        assert sorted(rid[b].tolist()) == list(range(N))
        assert np.all(np.diff(rsp[b]) <= 0)
        zero = rsp[b] == 0
        assert zero.any() and np.all(zero[np.argmax(zero):])  # the S' = 0 shapes close the row
        z = rid[b][zero]
        cand = dict(zip(ids[b].tolist(), sc[b].tolist()))
        is_c = np.array([p in cand for p in z])
        n_c = int(is_c.sum())
        assert is_c[:n_c].all() and not is_c[n_c:].any()  # candidates before unreached shapes
        s_c = np.array([cand[p] for p in z[:n_c]])
        assert np.all(np.diff(s_c) <= 0)
        assert np.all(np.diff(z[n_c:]) > 0)


@pytest.mark.parametrize("D", [256, 80])
def test_tensor_core_scan_tiling(gpu_lib, D):
    """BF16 store on the tcgen05 scan: buckets of >128 slots (several slot tiles),
    lists of >256 entries (several entry tiles), D with a partial 64-wide k-block;
    scan scores within BF16 error, rescored scores FP32-accurate."""
    import torch
    N, Nv, C, K = 100, 32, 2, 2
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 40, (64, 17), 91)
    ref = O.fif_scores(Q, qoff, qc, X, dbc)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="bf16", keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=N)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for b in range(len(qoff) - 1):
        assert sorted(ids[b].tolist()) == list(range(N))
        assert np.abs(sc[b] - ref[b, ids[b]]).max() < 3e-3
    ix.close()
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="bf16", rescore_r=N, keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=N)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for b in range(len(qoff) - 1):
        assert close(sc[b], ref[b, ids[b]]).all()
        assert_topk(ids[b], sc[b], ref[b], N)
    ix.close()


def test_rescore_depth_can_change_after_build(gpu_lib):
    """R = 0 on a rescoring index ranks by the store alone, like an index built without rescore;
    restoring R gives the built results again; an index without a rescore store refuses R > 0."""
    import torch
    N, Nv, D, C, K = 120, 16, 64, 4, 12
    X, cb, Q, qoff, dbc, qc = _case(N, Nv, D, C, K, 6, (16, 7), 121)
    q = torch.from_numpy(Q).cuda()
    with_r = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="bf16", rescore_r=30, keep_exact=False)
    no_r = _index(gpu_lib, torch, X, cb, N, Nv, K, storage="bf16", rescore_r=0, keep_exact=False)
    ref_i, ref_s = with_r.query(q, qoff, topk=10)
    with_r.set_rescore_depth(0)
    a = with_r.query(q, qoff, topk=10)
    b = no_r.query(q, qoff, topk=10)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    with_r.set_rescore_depth(30)
    c = with_r.query(q, qoff, topk=10)
    assert torch.equal(c[0], ref_i) and torch.equal(c[1], ref_s)
    with pytest.raises(gpu_lib.GiftError):
        no_r.set_rescore_depth(10)
    with pytest.raises(gpu_lib.GiftError):
        with_r.set_rescore_depth(2000)
    with_r.close()
    no_r.close()


@pytest.mark.parametrize("db_ma,q_ma,storage", [(2, 1, "f32"), (2, 2, "f32"), (3, 1, "bf16")])
def test_database_side_multiple_assignment(gpu_lib, db_ma, q_ma, storage):
    """Each database view enters db_ma lists (stored once per list): codes, lists and Eq. 4
    scores against the oracle with multiple assignment on the database side."""
    import torch
    N, Nv, D, C, K = 120, 16, 64, 4, 12
    X, cb, Q, qoff, _, _ = _case(N, Nv, D, C, K, 6, (16, 9), 131, ma=q_ma)
    R = 40 if storage != "f32" else 0
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage=storage, query_ma=q_ma, db_ma=db_ma, rescore_r=R,
                keep_exact=False)
    assert ix.info()["n_entries"] == N * Nv * db_ma
    codes, off, rows = ix.export_fif()
    rows_x = X.reshape(N * Nv, D)
    dbc = O.quantize(rows_x, cb, db_ma)
    assert_codes(codes.reshape(-1, db_ma), dbc, code_margins(rows_x, cb, db_ma))
    lists = O.build_fif(dbc.reshape(N, Nv, db_ma), K)
    for k, l in enumerate(lists):
        ref = (l[:, 0] * Nv + l[:, 1]) if len(l) else np.zeros(0, np.int64)
        assert np.array_equal(rows[off[k]:off[k + 1]], ref)
        assert np.all(np.diff(rows[off[k]:off[k + 1]]) > 0)  # a view enters a list once, in order
    ref = O.fif_scores(Q, qoff, O.quantize(Q, cb, q_ma), X, dbc.reshape(N, Nv, db_ma))
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=10)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for b in range(len(qoff) - 1):
        assert_topk(ids[b], sc[b], ref[b], 10)
    # the streamed build gives the same lists
    st = gpu_lib.Index.streamed(lambda f, n: X[f:f + n], torch.from_numpy(cb).cuda(), N, Nv, K, chunk_shapes=37,
                                storage=storage if storage != "f32" else "f32", query_ma=q_ma, rescore_r=R,
                                db_ma=db_ma)
    for a, b in zip(ix.export_fif(), st.export_fif()):
        assert np.array_equal(a, b)
    st.close()
    ix.close()


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_exact_match_from_the_list_store(gpu_lib, storage):
    """Eq. 3 on an index without the shape-ordered copy: the list-ordered two-part store is read
    once per query batch, FP32-level against the oracle."""
    import torch
    N, Nv, D, C, K = 90, 16, 64, 4, 8
    X, cb, Q, qoff, _, _ = _case(N, Nv, D, C, K, 7, (16, 5), 141)
    ix = _index(gpu_lib, torch, X, cb, N, Nv, K, storage=storage, rescore_r=20, keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="exact", topk=N)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    ref = O.exact_scores(Q, qoff, X)
    for b in range(len(qoff) - 1):
        assert_topk(ids[b], sc[b], ref[b], N)
    ix.close()
