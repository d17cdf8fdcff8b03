"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent brute force (explicit Python loops), a closed form worked by hand,
a special case where Eq. 4 must reduce to Eq. 3, an invariant, or finite
differences. A dropped term, a wrong index, sign or normaliser in the oracle
fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import shape_views, query_views, kmeans_codebook

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------- helpers
def py_cos(a, b):
    dot = sum(x * y for x, y in zip(a, b))
    na = math.sqrt(sum(x * x for x in a))
    nb = math.sqrt(sum(y * y for y in b))
    return 0.0 if na == 0 or nb == 0 else dot / (na * nb)


def py_exact(Q, q_off, X):
    """Eq. 3 by explicit loops over i, p, j."""
    N, Nv, _ = X.shape
    out = []
    for b in range(len(q_off) - 1):
        rows = [list(map(float, Q[i])) for i in range(q_off[b], q_off[b + 1])]
        out.append([sum(max(py_cos(q, list(map(float, X[p, j]))) for j in range(Nv)) for q in rows) / len(rows)
                    for p in range(N)])
    return np.array(out)


def py_codes(X, Bk, ma):
    """Nearest codewords by explicit squared differences, ties to the lower index."""
    out = []
    for x in X:
        d = [(sum((float(a) - float(c)) ** 2 for a, c in zip(x, b)), k) for k, b in enumerate(Bk)]
        d.sort()
        out.append([k for _, k in d[:ma]])
    return np.array(out)


def py_fif(Q, q_off, qc, X, dbc):
    """Eq. 4 by explicit loops: product with the Kronecker delta, max over all j
    (``dbc`` [N, N_v] or [N, N_v, m]: a database view matches through any of its codes)."""
    N, Nv, _ = X.shape
    dbc = np.asarray(dbc).reshape(N, Nv, -1)
    out = []
    for b in range(len(q_off) - 1):
        row = []
        for p in range(N):
            tot = 0.0
            for i in range(q_off[b], q_off[b + 1]):
                tot += max(py_cos(Q[i], X[p, j]) * (1.0 if set(dbc[p, j].tolist()) & set(qc[i].tolist()) else 0.0)
                           for j in range(Nv))
            row.append(tot / (q_off[b + 1] - q_off[b]))
        out.append(row)
    return np.array(out)


def rand_case(seed, N=5, Nv=4, D=6, B=3, signed=True, vq=(2, 3, 5)):
    g = np.random.default_rng(seed)
    X = g.standard_normal((N, Nv, D))
    counts = g.choice(vq, size=B)
    q_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    Q = g.standard_normal((q_off[-1], D))
    if not signed:
        X, Q = np.abs(X), np.abs(Q)
    return Q, q_off, X


# ----------------------------------------------------------------- cosine
def test_cosine_matches_explicit_loops_and_zero_norm():
    g = np.random.default_rng(0)
    A = g.standard_normal((4, 7))
    Bm = g.standard_normal((5, 7))
    A[2] = 0.0
    got = O.cosine(A, Bm)
    for i, j in itertools.product(range(4), range(5)):
        assert got[i, j] == pytest.approx(py_cos(A[i], Bm[j]), abs=1e-14)
    assert np.all(got[2] == 0.0)


def test_cosine_scale_invariance_and_self():
    g = np.random.default_rng(1)
    A = g.standard_normal((3, 9))
    assert np.allclose(np.diag(O.cosine(A, A)), 1.0, atol=1e-15)
    assert np.allclose(O.cosine(3.5 * A, 0.25 * A), O.cosine(A, A), atol=1e-15)


# ----------------------------------------------------------------- quantiser
@pytest.mark.parametrize("ma", [1, 2, 3])
def test_quantize_matches_brute_force(ma):
    g = np.random.default_rng(2 + ma)
    X = g.standard_normal((40, 3))
    Bk = g.standard_normal((6, 3))
    assert np.array_equal(O.quantize(X, Bk, ma), py_codes(X, Bk, ma))


def test_quantize_ties_go_to_lowest_index():
    Bk = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 0.0], [0.0, -1.0]])
    X = np.array([[1.0, 1.0], [2.0, 0.0], [0.0, 0.0]])
    # (1,1): d = 1,1,1,5 -> 0,1,2 ; (2,0): d = 1,5,1,5 -> 0,2,1 ; (0,0): all 1
    assert O.quantize(X, Bk, 1)[:, 0].tolist() == [0, 0, 0]
    assert O.quantize(X, Bk, 3).tolist() == [[0, 1, 2], [0, 2, 1], [0, 1, 2]]


# ----------------------------------------------------------------- hand-worked example
def test_hand_example_eq3_eq4():
    """Closed form worked by hand in 2-D.

    q = {(1,0), (0,1)}, p = {(1,1), (2,0), (0,-3)}; codebook (1,0), (0,1), (0,-1).
    Eq. 3: q1 -> max(1/sqrt2, 1, 0) = 1; q2 -> max(1/sqrt2, 0, -1) = 1/sqrt2;
           S = (1 + 1/sqrt2) / 2.
    Codes: q1 -> 0, q2 -> 1; p1 = (1,1) ties 0 and 1 -> 0; p2 -> 0; p3 -> 2.
    Eq. 4, MA=1: q1 meets p1, p2 -> 1; q2 meets nothing -> 0; S = 1/2.
    Eq. 4, MA=2: q1 -> {0, 1}, q2 -> {1, 0}; q2 meets p1, p2 -> 1/sqrt2;
           S = (1 + 1/sqrt2) / 2, equal to Eq. 3.
    """
    Q = np.array([[1.0, 0.0], [0.0, 1.0]])
    X = np.array([[[1.0, 1.0], [2.0, 0.0], [0.0, -3.0]]])
    Bk = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, -1.0]])
    off = np.array([0, 2])
    r2 = 1.0 / math.sqrt(2.0)
    assert O.exact_scores(Q, off, X)[0, 0] == pytest.approx((1 + r2) / 2, abs=1e-15)
    dbc = O.quantize(X.reshape(-1, 2), Bk, 1).reshape(1, 3)
    assert dbc.tolist() == [[0, 0, 2]]
    q1 = O.quantize(Q, Bk, 1)
    assert q1[:, 0].tolist() == [0, 1]
    assert O.fif_scores(Q, off, q1, X, dbc)[0, 0] == pytest.approx(0.5, abs=1e-15)
    q2 = O.quantize(Q, Bk, 2)
    assert q2.tolist() == [[0, 1], [1, 0]]
    assert O.fif_scores(Q, off, q2, X, dbc)[0, 0] == pytest.approx((1 + r2) / 2, abs=1e-15)
    lists = O.build_fif(dbc, 3)
    assert O.fif_scores_lists(Q, off, q1, X, lists)[0, 0] == pytest.approx(0.5, abs=1e-15)


# ----------------------------------------------------------------- Eq. 3 / Eq. 4 brute force
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_matches_brute_force(seed):
    Q, off, X = rand_case(seed)
    assert np.allclose(O.exact_scores(Q, off, X), py_exact(Q, off, X), atol=1e-13, rtol=0)


@pytest.mark.parametrize("seed,K,ma", [(0, 3, 1), (1, 4, 2), (2, 5, 3), (3, 2, 1)])
def test_fif_matches_brute_force_and_lists(seed, K, ma):
    Q, off, X = rand_case(seed, N=6, Nv=5, D=4)
    g = np.random.default_rng(100 + seed)
    Bk = g.standard_normal((K, 4))
    dbc = O.quantize(X.reshape(-1, 4), Bk, 1).reshape(6, 5)
    qc = O.quantize(Q, Bk, ma)
    lit = O.fif_scores(Q, off, qc, X, dbc)
    assert np.allclose(lit, py_fif(Q, off, qc, X, dbc), atol=1e-13, rtol=0)
    lists = O.build_fif(dbc, K)
    assert np.allclose(O.fif_scores_lists(Q, off, qc, X, lists), lit, atol=1e-13, rtol=0)


# ----------------------------------------------------------------- special cases of Eq. 4
@pytest.mark.parametrize("signed", [True, False])
def test_one_codeword_fif_equals_exact(signed):
    """K = 1: every delta is 1, so Eq. 4 is Eq. 3."""
    Q, off, X = rand_case(7, N=8, Nv=6, D=5, signed=signed)
    Bk = np.ones((1, 5))
    dbc = np.zeros((8, 6), np.int64)
    qc = O.quantize(Q, Bk, 1)
    ex = O.exact_scores(Q, off, X)
    assert np.allclose(O.fif_scores(Q, off, qc, X, dbc), ex, atol=1e-14, rtol=0)
    assert np.allclose(O.fif_scores_lists(Q, off, qc, X, O.build_fif(dbc, 1)), ex, atol=1e-13, rtol=0)


def test_full_multiple_assignment_equals_exact():
    """MA = K: every query view owns every codeword, so Eq. 4 is Eq. 3."""
    Q, off, X = rand_case(8, N=7, Nv=5, D=4)
    Bk = np.random.default_rng(9).standard_normal((4, 4))
    dbc = O.quantize(X.reshape(-1, 4), Bk, 1).reshape(7, 5)
    qc = O.quantize(Q, Bk, 4)
    assert np.allclose(O.fif_scores(Q, off, qc, X, dbc), O.exact_scores(Q, off, X), atol=1e-14, rtol=0)


def _small_mixture(n_shapes=30, nv=16, dim=24, classes=5, seed=11):
    X = shape_views(0, n_shapes, nv, dim, classes, 1000 + seed, 4000 + seed)
    Bk = kmeans_codebook(X.reshape(-1, dim), 12, 3000 + seed, 10)
    return X, Bk


def test_self_match_scores_one_and_ranks_first():
    X, Bk = _small_mixture()
    N, Nv, D = X.shape
    dbc = O.quantize(X.reshape(-1, D), Bk, 1).reshape(N, Nv)
    for p in (0, 7, 29):
        Q = X[p]
        off = np.array([0, Nv])
        qc = O.quantize(Q, Bk, 1)
        ex = O.exact_scores(Q, off, X)[0]
        fi = O.fif_scores(Q, off, qc, X, dbc)[0]
        assert ex[p] == pytest.approx(1.0, abs=1e-12)
        assert fi[p] == pytest.approx(1.0, abs=1e-12)
        assert O.rank(ex, 1)[0][0] == p and O.rank(fi, 1)[0][0] == p


def test_score_bounds_non_negative_features():
    """0 <= Eq.4 (MA=1) <= Eq.4 (MA=2) <= Eq.3 <= 1 for non-negative views."""
    X, Bk = _small_mixture(seed=12)
    N, Nv, D = X.shape
    Q, off, _ = query_views(4, (5, 9, 16), D, 5, 2012, 4012, max_views=16)
    dbc = O.quantize(X.reshape(-1, D), Bk, 1).reshape(N, Nv)
    f1 = O.fif_scores(Q, off, O.quantize(Q, Bk, 1), X, dbc)
    f2 = O.fif_scores(Q, off, O.quantize(Q, Bk, 2), X, dbc)
    ex = O.exact_scores(Q, off, X)
    eps = 1e-14
    assert np.all(f1 >= -eps) and np.all(f1 <= f2 + eps)
    assert np.all(f2 <= ex + eps) and np.all(ex <= 1 + eps)
    assert np.any(f1 < f2 - 1e-6)  # the pin is not vacuous


def test_posting_lists_partition_the_views():
    X, Bk = _small_mixture(seed=13)
    N, Nv, D = X.shape
    dbc = O.quantize(X.reshape(-1, D), Bk, 1).reshape(N, Nv)
    lists = O.build_fif(dbc, Bk.shape[0])
    allent = np.concatenate([l for l in lists if len(l)])
    assert len(allent) == N * Nv
    assert len({(int(p), int(j)) for p, j in allent}) == N * Nv
    for k, l in enumerate(lists):
        assert all(dbc[p, j] == k for p, j in l)
        keys = [int(p) * Nv + int(j) for p, j in l]
        assert keys == sorted(keys)


# ----------------------------------------------------------------- bounded top-k of Eq. 4
@pytest.mark.parametrize("signed,ma,k", [(False, 1, 5), (False, 2, 12), (True, 1, 7), (True, 2, 30)])
def test_bounded_topk_equals_full_ranking(signed, ma, k):
    """The pruned walk returns the top-k of the full Eq. 4 row (brute force over all shapes)."""
    if signed:
        Q, off, X = rand_case(21, N=40, Nv=6, D=8, B=4, signed=True, vq=(3, 6))
        Bk = np.random.default_rng(22).standard_normal((6, 8))
    else:
        X, Bk = _small_mixture(n_shapes=60, seed=14)
        Q, off, _ = query_views(4, (5, 9, 16), X.shape[2], 5, 2014, 4014, max_views=16)
        X, Q = X.astype(np.float64), Q.astype(np.float64)  # py_fif multiplies in the input type
    N, Nv, D = X.shape
    qc = O.quantize(Q, Bk, ma)
    full = py_fif(Q, off, qc, X, O.quantize(X.reshape(-1, D), Bk, 1).reshape(N, Nv))
    U = O.fif_upper_bound(Q, off, lambda f, n: X[f:f + n], N, chunk_shapes=7)
    assert np.all(full <= U + 1e-14)
    if not signed:  # all cosines >= 0: the bound is Eq. 3
        assert np.allclose(U, py_exact(Q, off, X), atol=1e-13, rtol=0)
    res, visited = O.fif_topk_bounded(Q, off, qc, Bk, lambda p: X[p], U, k, group=4)
    for b, (ids, sc) in enumerate(res):
        ref = O.rank(full[b], k)
        assert ids.tolist() == ref[0].tolist()
        assert np.allclose(sc, ref[1], atol=1e-13, rtol=0)
    if not signed:
        assert min(visited) < N  # the bound prunes on clustered views


def test_bounded_topk_bound_uses_zero_candidate():
    """A query view whose cosines are all negative still bounds Eq. 4 by 0, not by its max."""
    X = -np.ones((3, 2, 2))
    X[2, 0] = [1.0, 0.0]
    Q = np.array([[1.0, 0.0], [0.0, 1.0]])
    off = np.array([0, 2])
    U = O.fif_upper_bound(Q, off, lambda f, n: X[f:f + n], 3)
    assert U[0].tolist() == pytest.approx([0.0, 0.0, 0.5])
    res, _ = O.fif_topk_bounded(Q, off, np.array([[0], [0]]), np.ones((1, 2)), lambda p: X[p], U, 3)
    assert res[0][0].tolist() == [2, 0, 1]


# ----------------------------------------------------------------- counter generator
def test_counter_generator_host_and_torch_bit_identical():
    torch = pytest.importorskip("torch")
    from synth.counter import shape_views_np, shape_views_torch
    a = shape_views_np(13, 5, 7, 48, 3, 77, 78)
    b = shape_views_torch(13, 5, 7, 48, 3, 77, 78, device="cpu").numpy()
    assert a.dtype == np.float32 and np.array_equal(a, b)
    assert np.array_equal(shape_views_np(15, 1, 7, 48, 3, 77, 78)[0], a[2])  # any range alone
    assert np.all(a >= 0) and np.allclose(np.linalg.norm(a, axis=2), 1.0, atol=1e-6)


def test_counter_generator_splitmix64_reference_values():
    """splitmix64 seeded with 0: its published first outputs."""
    from synth.counter import _mix_np, _GOLDEN
    z = (np.arange(1, 4, dtype=np.uint64) * np.uint64(_GOLDEN))
    got = [int(v) for v in _mix_np(z)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ----------------------------------------------------------------- ranking
def test_rank_matches_sorted_with_ties():
    s = np.array([0.3, 0.9, 0.3, 0.1, 0.9, 0.0, 0.3])
    ids, vals = O.rank(s, 5)
    ref = sorted(range(len(s)), key=lambda i: (-s[i], i))[:5]
    assert ids.tolist() == ref == [1, 4, 0, 2, 6]
    assert vals.tolist() == [s[i] for i in ref]


# ----------------------------------------------------------------- S-IF (Eqs. 5-8, 12-14)
def test_membership_vector_eq7():
    s = np.array([0.2, 0.8, 0.5, 0.8, 0.1])
    F = O.membership(s, 3)
    assert F.tolist() == [0.0, 0.8, 0.5, 0.8, 0.0]


def test_membership_of_negative_scores_is_zero():
    """A neighbour with a negative score (signed features) has membership 0: worked by hand,
    the first four of the ranking are shapes 1, 3, 4, 0 and only 1 and 3 score above 0."""
    s = np.array([-0.1, 0.9, -0.3, 0.4, -0.05])
    assert O.membership(s, 4).tolist() == [0.0, 0.9, 0.0, 0.4, 0.0]
    # Eq. 8 on such activations, scores +-1: the crisp Jaccard index of {1, 3} and {0, 3, 4}
    Fa = O.membership(np.array([-1.0, 1.0, -1.0, 1.0, -0.5]), 4)
    assert Fa.tolist() == [0.0, 1.0, 0.0, 1.0, 0.0]
    assert O.contextual(Fa, np.array([1.0, 0.0, 0.0, 1.0, 1.0])) == pytest.approx(1 / 4, abs=1e-15)


def test_contextual_reduces_to_crisp_jaccard():
    """With all memberships 1, Eq. 8 is the set Jaccard index of Eq. 5."""
    g = np.random.default_rng(3)
    for _ in range(20):
        a = set(g.choice(30, 8, replace=False).tolist())
        b = set(g.choice(30, 8, replace=False).tolist())
        Fa = np.zeros(30)
        Fb = np.zeros(30)
        Fa[list(a)] = 1.0
        Fb[list(b)] = 1.0
        assert O.contextual(Fa, Fb) == pytest.approx(len(a & b) / len(a | b), abs=1e-15)


def test_contextual_properties():
    g = np.random.default_rng(4)
    for _ in range(20):
        Fa = np.where(g.random(25) < 0.3, g.random(25), 0.0)
        Fb = np.where(g.random(25) < 0.3, g.random(25), 0.0)
        v = O.contextual(Fa, Fb)
        assert 0.0 <= v <= 1.0
        assert v == pytest.approx(O.contextual(Fb, Fa), abs=1e-15)
        if Fa.any():
            assert O.contextual(Fa, Fa) == pytest.approx(1.0, abs=1e-15)
        # explicit loops of Eq. 6 over the union / intersection of supports
        inter = [i for i in range(25) if Fa[i] > 0 and Fb[i] > 0]
        union = [i for i in range(25) if Fa[i] > 0 or Fb[i] > 0]
        ref = (sum(min(Fa[i], Fb[i]) for i in inter) / sum(max(Fa[i], Fb[i]) for i in union)) if union else 0.0
        assert v == pytest.approx(ref, abs=1e-14)
    assert O.contextual(np.zeros(4), np.zeros(4)) == 0.0


def test_inverted_file_route_equals_dense_eq8():
    X, Bk = _small_mixture(n_shapes=40, seed=14)
    N, Nv, D = X.shape
    dbc = O.quantize(X.reshape(-1, D), Bk, 1).reshape(N, Nv)
    S_db = O.fif_scores(X.reshape(-1, D), np.arange(0, N * Nv + 1, Nv), O.quantize(X.reshape(-1, D), Bk, 1), X, dbc)
    F_db = O.db_memberships(S_db, 6)
    # self is in every database neighbour set
    assert all(F_db[p, p] > 0 for p in range(N))
    card, entries = O.build_sif(F_db)
    assert sum(len(e[0]) for e in entries) == N * 6
    Q, off, _ = query_views(5, (16,), D, 5, 2014, 4014, max_views=16)
    S_q = O.fif_scores(Q, off, O.quantize(Q, Bk, 1), X, dbc)
    for b in range(5):
        Fq = O.membership(S_q[b], 6)
        dense = np.array([O.contextual(Fq, F_db[p]) for p in range(N)])
        inv = O.sif_scores_inverted(Fq, card, entries)
        assert np.allclose(inv, dense, atol=1e-14, rtol=0)


def test_rerank_order_brute_force():
    g = np.random.default_rng(5)
    N = 12
    S_db = g.random((N, N))
    np.fill_diagonal(S_db, 1.0)
    F_db = O.db_memberships(S_db, 4)
    S_q = g.random((2, N))
    ids, sp = O.rerank(S_q, F_db, 4, 6)
    for b in range(2):
        Fq = O.membership(S_q[b], 4)
        spv = [O.contextual(Fq, F_db[p]) for p in range(N)]
        ref = sorted(range(N), key=lambda p: (-spv[p], -S_q[b, p], p))[:6]
        assert ids[b].tolist() == ref


# ----------------------------------------------------------------- differentiation
def _tie_free(seed, B=2, Np=4, nv=8, din=16, dout=6, margin=1e-3):
    g = np.random.default_rng(seed)
    while True:
        Q = g.standard_normal((B * nv, din))
        P = g.standard_normal((Np, nv, din))
        W = g.standard_normal((dout, din)) / 4
        U = Q @ W.T
        V = P.reshape(-1, din) @ W.T
        s = O.cosine(U, V).reshape(B * nv, Np, nv)
        top2 = np.sort(s, axis=2)[:, :, -2:]
        if np.min(top2[:, :, 1] - top2[:, :, 0]) > margin:
            return Q, np.arange(0, B * nv + 1, nv), P, W, g.standard_normal((B, Np))


def test_backward_matches_central_differences():
    Q, off, P, W, G = _tie_free(21)
    dW, dQ, dP = O.match_backward(Q, off, P, W, G)
    h = 1e-6

    def L(Q_, P_, W_):
        return float((O.match_forward(Q_, off, P_, W_)[0] * G).sum())

    g = np.random.default_rng(0)
    for _ in range(12):
        i, d = g.integers(Q.shape[0]), g.integers(Q.shape[1])
        Qp, Qm = Q.copy(), Q.copy()
        Qp[i, d] += h
        Qm[i, d] -= h
        assert dQ[i, d] == pytest.approx((L(Qp, P, W) - L(Qm, P, W)) / (2 * h), abs=2e-7)
        p, j, d = g.integers(P.shape[0]), g.integers(P.shape[1]), g.integers(P.shape[2])
        Pp, Pm = P.copy(), P.copy()
        Pp[p, j, d] += h
        Pm[p, j, d] -= h
        assert dP[p, j, d] == pytest.approx((L(Q, Pp, W) - L(Q, Pm, W)) / (2 * h), abs=2e-7)
        r, c = g.integers(W.shape[0]), g.integers(W.shape[1])
        Wp, Wm = W.copy(), W.copy()
        Wp[r, c] += h
        Wm[r, c] -= h
        assert dW[r, c] == pytest.approx((L(Q, P, Wp) - L(Q, P, Wm)) / (2 * h), abs=2e-7)


def test_backward_scale_invariants():
    """Cosine is scale-invariant: <q_i, dS/dq_i> = 0, <p_j, dS/dp_j> = 0, <W, dS/dW> = 0."""
    Q, off, P, W, G = _tie_free(22)
    dW, dQ, dP = O.match_backward(Q, off, P, W, G)
    assert np.allclose((Q * dQ).sum(1), 0.0, atol=1e-12)
    assert np.allclose((P * dP).sum(2), 0.0, atol=1e-12)
    assert abs((W * dW).sum()) < 1e-12
    assert np.abs(dQ).max() > 1e-3  # not vacuous


def test_backward_identity_projection():
    Q, off, P, W, G = _tie_free(23, dout=16)
    _, dQ0, dP0 = O.match_backward(Q, off, P, None, G)
    _, dQ1, dP1 = O.match_backward(Q, off, P, np.eye(16), G)
    assert np.allclose(dQ0, dQ1, atol=1e-14) and np.allclose(dP0, dP1, atol=1e-14)
    S0, j0 = O.match_forward(Q, off, P, None)
    assert np.allclose(S0, O.exact_scores(Q, off, P), atol=1e-14)


# ----------------------------------------------------------------- two measures: Eqs. 9-11
def _score_matrix(g, N, ties=False):
    S = g.random((N, N))
    if ties:
        S = np.round(S, 1)
    np.fill_diagonal(S, 1.0)  # a database shape matched with itself scores 1 (self-match)
    return S


def py_genmean(a, b, alpha):
    return ((a ** alpha + b ** alpha) / 2.0) ** (1.0 / alpha)


def py_aca(S1, S2, F1_db, F2_db, k1, k2, alpha, mode):
    """ACA by explicit loops: sorted neighbour lists, per-coordinate sums, Eq. 9 per coordinate."""
    N = len(S1)

    def first(S, k):
        return [i for _, i in sorted((-S[i], i) for i in range(N))[:k]]

    def eq7(S):
        F = [0.0] * N
        for i in first(S, k1):
            F[i] = float(S[i])
        return F

    def mean_rows(F, nbrs):
        return [sum(F[i][j] for i in nbrs) / len(nbrs) for j in range(N)]

    if mode == "none":
        A1, A2 = eq7(S1), eq7(S2)
    elif mode == "aug":
        A1, A2 = mean_rows(F1_db, first(S1, k2)), mean_rows(F2_db, first(S2, k2))
    else:
        A1, A2 = mean_rows(F1_db, first(S2, k2)), mean_rows(F2_db, first(S1, k2))
    return [py_genmean(a, b, alpha) for a, b in zip(A1, A2)]


def test_generalised_mean_eq9_closed_forms():
    a = np.array([0.0, 0.25, 0.5, 1.0, 0.9])
    b = np.array([0.0, 0.0, 0.5, 0.04, 0.1])
    assert np.allclose(O.aca_fuse(a, b, 1.0), (a + b) / 2, atol=1e-15)
    assert np.allclose(O.aca_fuse(a, b, 0.5), ((np.sqrt(a) + np.sqrt(b)) / 2) ** 2, atol=1e-15)
    assert np.allclose(O.aca_fuse(a, a, 0.5), a, atol=1e-15) and np.allclose(O.aca_fuse(b, b, 0.3), b, atol=1e-15)
    f = O.aca_fuse(a, b, 0.5)
    assert np.all(f >= np.minimum(a, b) - 1e-15) and np.all(f <= np.maximum(a, b) + 1e-15)
    assert f[1] == pytest.approx(0.25 / 4)  # one activation zero: (sqrt(a)/2)^2


@pytest.mark.parametrize("mode,alpha,k1,k2", [("none", 0.5, 4, 2), ("aug", 0.5, 5, 3), ("co", 0.5, 5, 3),
                                              ("co", 1.0, 3, 2), ("co", 0.5, 6, 1)])
def test_aca_matches_loops(mode, alpha, k1, k2):
    g = np.random.default_rng(31)
    N = 12
    S1_db, S2_db = _score_matrix(g, N), _score_matrix(g, N)
    S1_q, S2_q = g.random(N), g.random(N)
    F1_db, F2_db = O.db_memberships(S1_db, k1), O.db_memberships(S2_db, k1)
    got = O.aca_activation(S1_q, S2_q, F1_db, F2_db, k1, k2, alpha, mode)
    ref = py_aca(list(S1_q), list(S2_q), F1_db.tolist(), F2_db.tolist(), k1, k2, alpha, mode)
    assert np.allclose(got, ref, atol=1e-15)
    A = O.aca_db(S1_db, S2_db, k1, k2, alpha, mode)
    for p in (0, 7):
        assert np.allclose(A[p], py_aca(list(S1_db[p]), list(S2_db[p]), F1_db.tolist(), F2_db.tolist(), k1, k2,
                                        alpha, mode), atol=1e-15)


def test_aca_reduces_to_one_measure():
    """Equal measures make Eq. 9 the identity: ACA without augmentation is Eq. 7, co-augmentation is
    augmentation, and with k2 = 1 a database shape's augmented activation is its own (self ranks first)."""
    g = np.random.default_rng(32)
    N, k1 = 15, 5
    S_db = _score_matrix(g, N)
    S_q = g.random((3, N))
    F_db = O.db_memberships(S_db, k1)
    for b in range(3):
        assert np.allclose(O.aca_activation(S_q[b], S_q[b], F_db, F_db, k1, 4, 0.5, "none"),
                           O.membership(S_q[b], k1), atol=1e-15)
        assert np.allclose(O.aca_activation(S_q[b], S_q[b], F_db, F_db, k1, 4, 0.5, "co"),
                           O.aca_activation(S_q[b], S_q[b], F_db, F_db, k1, 4, 0.5, "aug"), atol=1e-15)
    assert np.allclose(O.aca_db(S_db, S_db, k1, 1, 0.5, "aug"), F_db, atol=1e-15)
    ids_a, sp_a = O.rerank_aca(S_q, S_q, S_db, S_db, k1, 4, 0.5, "none", 8)
    ids_r, sp_r = O.rerank(S_q, F_db, k1, 8)
    assert np.array_equal(ids_a, ids_r) and np.allclose(sp_a, sp_r, atol=1e-15)


def test_aca_inverted_route_equals_dense_eq8():
    """ACA activations are non-negative, so Eq. 13/14 through the second inverted file give Eq. 8."""
    g = np.random.default_rng(33)
    N = 14
    S1_db, S2_db = _score_matrix(g, N, ties=True), _score_matrix(g, N, ties=True)
    A = O.aca_db(S1_db, S2_db, 4, 2, 0.5, "co")
    assert np.all(A >= 0) and np.all((A > 0).sum(axis=1) <= 2 * 2 * 4)
    card, entries = O.build_sif(A)
    F1_db, F2_db = O.db_memberships(S1_db, 4), O.db_memberships(S2_db, 4)
    Fq = O.aca_activation(g.random(N), g.random(N), F1_db, F2_db, 4, 2, 0.5, "co")
    inv = O.sif_scores_inverted(Fq, card, entries)
    dense = np.array([O.contextual(Fq, A[p]) for p in range(N)])
    assert np.allclose(inv, dense, atol=1e-14)


# ----------------------------------------------------------------- k-means vocabulary
def py_lloyd(X, init, iters):
    X = [list(map(float, r)) for r in X]
    C = [list(X[i]) for i in init]
    for _ in range(iters):
        lab, dist = [], []
        for x in X:
            ds = [(sum((a - b) ** 2 for a, b in zip(x, c)), k) for k, c in enumerate(C)]
            d, k = min(ds)
            lab.append(k)
            dist.append(d)
        far = [i for _, i in sorted((-d, i) for i, d in enumerate(dist))]
        fi, newC = 0, []
        for c in range(len(C)):
            rows = [i for i, l in enumerate(lab) if l == c]
            if rows:
                newC.append([sum(X[i][d] for i in rows) / len(rows) for d in range(len(X[0]))])
            else:
                newC.append(list(X[far[fi]]))
                fi += 1
        C = newC
    return np.array(C)


def test_lloyd_matches_loops_and_reseeds_empty_centres():
    g = np.random.default_rng(41)
    X = g.standard_normal((40, 3))
    assert np.allclose(O.kmeans_lloyd(X, [0, 5, 9, 13], 4), py_lloyd(X, [0, 5, 9, 13], 4), atol=1e-12)
    # a duplicated initial centre leaves the second copy empty: it takes the farthest row
    Y = np.array([[0.0, 0], [0, 1], [10, 0], [10, 1], [50, 50]])
    C = O.kmeans_lloyd(Y, [0, 0, 2], 1)
    assert np.allclose(C, py_lloyd(Y, [0, 0, 2], 1))
    assert np.allclose(C[1], [50, 50]) and np.allclose(C[0], [0, 0.5])


def test_lloyd_separated_blobs_and_monotone_objective():
    g = np.random.default_rng(42)
    centres = np.array([[0.0, 0, 0], [20, 0, 0], [0, 20, 0]])
    X = np.concatenate([c + g.standard_normal((30, 3)) for c in centres])
    C = O.kmeans_lloyd(X, [0, 30, 60], 3)
    for b in range(3):
        assert np.allclose(C[b], X[30 * b:30 * (b + 1)].mean(axis=0), atol=1e-12)
    obj = []
    for it in range(5):
        Ck = O.kmeans_lloyd(X, [0, 1, 2], it)
        lab = O.quantize(X, Ck, 1)[:, 0]
        obj.append(((X - Ck[lab]) ** 2).sum())
    assert all(b <= a + 1e-9 for a, b in zip(obj, obj[1:]))


# ----------------------------------------------------------------- database-side multiple assignment
@pytest.mark.parametrize("seed,K,ma_q,ma_db", [(0, 4, 1, 2), (1, 5, 2, 2), (2, 6, 1, 3)])
def test_database_side_multiple_assignment(seed, K, ma_q, ma_db):
    Q, off, X = rand_case(seed, N=6, Nv=5, D=4)
    Bk = np.random.default_rng(200 + seed).standard_normal((K, 4))
    dbc = O.quantize(X.reshape(-1, 4), Bk, ma_db).reshape(6, 5, ma_db)
    qc = O.quantize(Q, Bk, ma_q)
    lit = O.fif_scores(Q, off, qc, X, dbc)
    assert np.allclose(lit, py_fif(Q, off, qc, X, dbc), atol=1e-13, rtol=0)
    lists = O.build_fif(dbc, K)
    assert sum(len(l) for l in lists) == 6 * 5 * ma_db
    assert np.allclose(O.fif_scores_lists(Q, off, qc, X, lists), lit, atol=1e-13, rtol=0)
    # more database assignments can only add matches
    assert np.all(lit >= O.fif_scores(Q, off, qc, X, dbc[..., :1]) - 1e-15)


def test_database_side_full_assignment_equals_exact():
    """m = K on the database side: every view is in every list, so Eq. 4 is Eq. 3."""
    Q, off, X = rand_case(9, N=5, Nv=4, D=3)
    Bk = np.random.default_rng(10).standard_normal((3, 3))
    dbc = O.quantize(X.reshape(-1, 3), Bk, 3).reshape(5, 4, 3)
    assert np.allclose(O.fif_scores(Q, off, O.quantize(Q, Bk, 1), X, dbc), O.exact_scores(Q, off, X),
                       atol=1e-14, rtol=0)


# ----------------------------------------------------------------- projection rendering (Sec. 2.1)
def py_raster(S, T, H, W):
    """Depth buffer by explicit loops over pixels and triangles (closed triangles, nearest depth)."""
    D = [[2.0] * W for _ in range(H)]
    for i in range(H):
        for j in range(W):
            px, py = -1 + (2 * j + 1) / W, 1 - (2 * i + 1) / H
            for t in T:
                (ax, ay, az), (bx, by, bz), (cx, cy, cz) = (S[k] for k in t)
                area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
                if area == 0:
                    continue
                w = [(cx - bx) * (py - by) - (cy - by) * (px - bx), (ax - cx) * (py - cy) - (ay - cy) * (px - cx),
                     (bx - ax) * (py - ay) - (by - ay) * (px - ax)]
                if area < 0:
                    w = [-x for x in w]
                    area = -area
                if min(w) >= 0:
                    D[i][j] = min(D[i][j], (w[0] * az + w[1] * bz + w[2] * cz) / area)
    return np.array(D)


def test_raster_half_screen_and_zbuffer():
    # the lower-left half-screen triangle at depth 0.5 over a full-screen pair at depth 1.0
    S = np.array([[-1, -1, 0.5], [1, -1, 0.5], [-1, 1, 0.5], [-1, -1, 1.0], [1, -1, 1.0], [1, 1, 1.0], [-1, 1, 1.0]])
    T = np.array([[0, 1, 2], [3, 4, 5], [3, 5, 6]])
    D = O.raster_depth(S, T, 4, 4)
    X, Y = np.meshgrid(-1 + (2 * np.arange(4) + 1) / 4, 1 - (2 * np.arange(4) + 1) / 4)
    assert np.array_equal(D, np.where(X + Y <= 0, 0.5, 1.0))
    g = np.random.default_rng(51)
    S = np.concatenate([g.uniform(-1.2, 1.2, (9, 2)), g.uniform(0, 2, (9, 1))], axis=1)
    T = g.integers(0, 9, (6, 3))
    assert np.allclose(O.raster_depth(S, T, 7, 9), py_raster(S, T, 7, 9), atol=1e-12)


def test_normalisation_invariance_and_frames():
    from synth.meshes import star_mesh
    V, T = star_mesh(4, 3, 9, n_lat=8, n_lon=12)
    c, s = O.normalize_mesh(V, T)
    P = (V - c) * s
    assert np.sqrt((P ** 2).sum(1)).max() == pytest.approx(1.0)
    c2, s2 = O.normalize_mesh(P, T)
    assert np.allclose(c2, 0, atol=1e-12) and s2 == pytest.approx(1.0)
    a = O.render_depth(V, T, 4, 2, 12, 12)
    b = O.render_depth(V.astype(np.float64) * 3.5 + np.array([7.0, -2, 5]), T, 4, 2, 12, 12)
    assert np.allclose(a, b, atol=1e-9)
    C, f, r, u = O.view_frames(8, 8)
    assert np.allclose(np.linalg.norm(C, axis=1), 1) and np.allclose((r * f).sum(1), 0)
    assert np.allclose(np.cross(r, u), -f)  # right-handed: r x u points back at the camera


def test_sphere_depth_closed_form():
    """A finely tessellated sphere: the silhouette covers the disc x^2 + y^2 <= 1 and the
    front surface lies at depth 1 - sqrt(1 - x^2 - y^2)."""
    n_lat, n_lon = 64, 128
    th = np.pi * np.arange(1, n_lat) / n_lat
    ph = 2 * np.pi * np.arange(n_lon) / n_lon
    TT, PP = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([np.sin(TT) * np.cos(PP), np.sin(TT) * np.sin(PP), np.cos(TT)], -1).reshape(-1, 3)
    V = np.concatenate([[[0, 0, 1.0]], ring, [[0, 0, -1.0]]])
    idx = lambda i, j: 1 + i * n_lon + (j % n_lon)
    T = [(0, idx(0, j), idx(0, j + 1)) for j in range(n_lon)]
    T += [(len(V) - 1, idx(n_lat - 2, j + 1), idx(n_lat - 2, j)) for j in range(n_lon)]
    for i in range(n_lat - 2):
        for j in range(n_lon):
            T += [(idx(i, j), idx(i + 1, j), idx(i, j + 1)), (idx(i, j + 1), idx(i + 1, j), idx(i + 1, j + 1))]
    D = O.render_depth(V, np.array(T), 2, 1, 16, 16)[0]
    X, Y = np.meshgrid(-1 + (2 * np.arange(16) + 1) / 16, 1 - (2 * np.arange(16) + 1) / 16)
    R2 = X ** 2 + Y ** 2
    inner = R2 < 0.85
    assert np.all(D[inner] < 2) and np.all(D[R2 > 1.05] == 2)
    assert np.abs(D[inner] - (1 - np.sqrt(1 - R2[inner]))).max() < 5e-3
