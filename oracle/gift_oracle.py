"""FP64 CPU oracle of GIFT's on-line query path (Bai et al., GIFT, CVPR 2016).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or call this
module; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it. It shares no code with the CUDA library.

Every float is widened to float64. Loops are plain; numpy matrix products serve
as library steps. What each function computes, with the passage it follows:

* ``cosine``               s(a, b), the cosine similarity used in Eq. 3 (Sec. 2.3)
* ``quantize``             c(x) = argmin_k ||x - b_k||^2 (Sec. 2.3, after Eq. 4),
                           with multiple assignment (Sec. 2.3, last paragraph)
* ``kmeans_lloyd``         the off-line vocabulary: Lloyd's k-means (Sec. 2.3)
* ``build_fif``            the first inverted file (Sec. 2.3, Fig. 2)
* ``exact_scores``         S(x_q, x_p), Eq. 3
* ``fif_scores``           the approximate match of Eq. 4, literally (Kronecker delta)
* ``fif_scores_lists``     Eq. 4 evaluated by walking the inverted file
* ``fif_upper_bound``/``fif_topk_bounded``  the top-k of Eq. 4 over a database
                           too large to quantise whole: an upper bound of every
                           Eq. 4 term prunes the shapes that cannot rank
* ``normalize_mesh``/``view_frames``/``raster_depth``/``render_depth``  the
                           projection front end of Sec. 2.1: scale and translation
                           normalisation, cameras on the unit sphere by azimuth and
                           elevation, depth-buffer views
* ``rank``                 the ranked list, order (score desc, id asc)
* ``membership``           the sparse activation F_q of Eq. 7
* ``contextual``           S'(x_q, x_p) of Eq. 8
* ``build_sif``/``sif_scores_inverted``  Eq. 13 / Eq. 14 over the second
                           inverted file (Sec. 2.4.2, Fig. 3)
* ``rerank``               the re-ranked list by (S' desc, S desc, id asc)
* ``augment``/``aca_fuse``/``aca_activation``/``rerank_aca``  two similarity
                           measures: neighbour augmentation (Eq. 10), co-augmentation
                           (Eq. 11), the generalised-mean aggregation of Eq. 9 and the
                           re-rank by S' of the fused activations
* ``match_forward``/``match_backward``  Eq. 3 after a linear view projection
                           u = W q, and its gradient through the argmax view

Readings where the paper is silent (each also listed in the design notes):
* the normaliser of Eq. 3/4 is the query's own view count |V(x_q)|;
* Eq. 4 is taken literally: the max runs over all database views, so a view
  whose code differs contributes a 0 candidate;
* quantiser ties go to the lowest codeword index; multiple assignment returns
  the m nearest codewords ordered by (distance, index); database views use one
  assignment, queries ``ma``;
* ranking ties go to the lower shape id; re-ranking orders by
  (S' desc, S desc, id asc); S' = 0 when both F vectors are zero;
* an Eq. 7 membership is the positive part of the neighbour's score (a
  negative score, possible only with signed features, gives membership 0);
* a database shape's neighbour set N_k1 includes the shape itself;
* rendering: the centroid is the area-weighted surface centroid; cameras use
  orthographic projection along the view axis (the image plane spans the unit
  sphere's silhouette), elevations avoid the poles, and a pixel samples its
  centre with closed triangles (edge functions >= 0);
* with two measures, the re-ranked order breaks S' ties by the first measure's
  score S^(1), then by id; the neighbour sets of Eqs. 10/11 are the first k2
  entries of the same rankings that give N_k1;
* the squared distance is evaluated as ||x||^2 - 2 x.b + ||b||^2 in float64
  (an algebraic identity; its rounding, about 1e-15 of ||x||^2 + ||b||^2,
  is far below any margin at which codes are compared).

Parity pins for every function are in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import numpy as np

# rows of the database processed per float64 chunk (bounds host memory)
_CHUNK_ROWS = 8192


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def cosine(A, B):
    """Matrix of s(a_i, b_j) = a_i . b_j / (||a_i|| ||b_j||); 0 when a norm is 0.

    The similarity s of Eq. 3 is the cosine (Sec. 2.3, sentence after Eq. 3).
    """
    A = _f64(A)
    B = _f64(B)
    na = np.sqrt((A * A).sum(axis=1))
    nb = np.sqrt((B * B).sum(axis=1))
    G = A @ B.T
    den = np.outer(na, nb)
    out = np.zeros_like(G)
    nz = den > 0
    out[nz] = G[nz] / den[nz]
    return out


def sq_distances(X, Bk):
    """||x_i - b_k||^2 for all pairs, float64 [n, K] (expanded form, see header)."""
    X = _f64(X)
    Bk = _f64(Bk)
    xx = (X * X).sum(axis=1)
    bb = (Bk * Bk).sum(axis=1)
    return xx[:, None] - 2.0 * (X @ Bk.T) + bb[None, :]


def quantize(X, codebook, ma=1):
    """Codes int64 [n, ma]: the ma nearest codewords of each row, by (distance, index).

    c(x) = argmin_{1<=i<=K} ||x - b_i||^2 (Sec. 2.3); multiple assignment keeps
    several nearest codewords (Sec. 2.3, last paragraph).
    """
    X = _f64(X)
    out = np.empty((X.shape[0], ma), np.int64)
    for lo in range(0, X.shape[0], _CHUNK_ROWS):
        d = sq_distances(X[lo:lo + _CHUNK_ROWS], codebook)
        # a stable sort on distance puts equal distances in index order
        out[lo:lo + _CHUNK_ROWS] = np.argsort(d, axis=1, kind="stable")[:, :ma]
    return out


def kmeans_lloyd(X, init_rows, iters):
    """Lloyd's k-means for the vocabulary B of Sec. 2.3 (trained off-line with
    k-means; the paper gives no details), float64 [K, D].

    Starts from the rows ``init_rows``; each iteration assigns every row to its
    nearest centre (``quantize``: ties to the lowest index) and moves each centre
    to the mean of its rows. A centre left without rows takes the row farthest
    from the centre it was assigned to in that iteration (rows by distance
    desc, index asc), the empty centres served in ascending order.
    """
    X = _f64(X)
    C = X[np.asarray(init_rows, np.int64)].copy()
    K = C.shape[0]
    for _ in range(iters):
        lab = quantize(X, C, 1)[:, 0]
        d = ((X - C[lab]) ** 2).sum(axis=1)
        far = np.lexsort((np.arange(X.shape[0]), -d))
        fi = 0
        newC = C.copy()
        for c in range(K):
            rows = np.nonzero(lab == c)[0]
            if len(rows):
                newC[c] = X[rows].sum(axis=0) / len(rows)
            else:
                newC[c] = X[far[fi]]
                fi += 1
        C = newC
    return C


def build_fif(db_codes, n_codewords):
    """First inverted file (Fig. 2): list k holds every (shape, view) with k among its codes.

    ``db_codes`` is int [N, N_v] (one assignment per database view) or
    [N, N_v, m] (database-side multiple assignment: a view enters m lists, at
    the memory cost Sec. 2.3 mentions). Each list is in ascending (shape, view)
    order. Returns a list of K int64 arrays of shape [L_k, 2].
    """
    db_codes = np.asarray(db_codes)
    N, Nv = db_codes.shape[:2]
    codes = db_codes.reshape(N, Nv, -1)
    lists = [[] for _ in range(n_codewords)]
    for p in range(N):
        for j in range(Nv):
            for c in codes[p, j]:
                lists[int(c)].append((p, j))
    return [np.asarray(l, np.int64).reshape(-1, 2) for l in lists]


def _db_rows(X):
    X = np.asarray(X)
    N, Nv, D = X.shape
    return X.reshape(N * Nv, D), N, Nv


def exact_scores(Q, q_off, X):
    """Eq. 3: S(x_q, x_p) = (1/|V(x_q)|) sum_i max_j s(q_i, p_j), float64 [B, N]."""
    rows, N, Nv = _db_rows(X)
    q_off = np.asarray(q_off)
    B = len(q_off) - 1
    S = np.zeros((B, N))
    for b in range(B):
        Qb = _f64(Q[q_off[b]:q_off[b + 1]])
        V = Qb.shape[0]
        for lo in range(0, N, max(1, _CHUNK_ROWS // Nv)):
            hi = min(N, lo + max(1, _CHUNK_ROWS // Nv))
            s = cosine(Qb, rows[lo * Nv:hi * Nv]).reshape(V, hi - lo, Nv)
            S[b, lo:hi] = s.max(axis=2).sum(axis=0) / V
    return S


def fif_scores(Q, q_off, q_codes, X, db_codes):
    """Eq. 4 taken literally, float64 [B, N].

    S(x_q, x_p) = (1/|V(x_q)|) sum_i max_j s(q_i, p_j) * delta(c(q_i), c(p_j)),
    where delta is 1 when q_i's assigned codewords and p_j's share a codeword
    (multiple assignment, Sec. 2.3, on either side: ``db_codes`` is [N, N_v] or
    [N, N_v, m]) and 0 otherwise. The max runs over all j, so an unmatched view
    contributes the candidate value 0.
    """
    rows, N, Nv = _db_rows(X)
    dbc = np.asarray(db_codes).reshape(N, Nv, -1)
    q_codes = np.asarray(q_codes)
    q_off = np.asarray(q_off)
    B = len(q_off) - 1
    S = np.zeros((B, N))
    step = max(1, _CHUNK_ROWS // Nv)
    for b in range(B):
        Qb = _f64(Q[q_off[b]:q_off[b + 1]])
        cb = q_codes[q_off[b]:q_off[b + 1]]
        V = Qb.shape[0]
        for lo in range(0, N, step):
            hi = min(N, lo + step)
            s = cosine(Qb, rows[lo * Nv:hi * Nv]).reshape(V, hi - lo, Nv)
            # delta[i, p, j] = 1 iff a codeword of p_j is among q_i's codewords
            delta = (dbc[None, lo:hi, :, :, None] == cb[:, None, None, None, :]).any(axis=(3, 4))
            S[b, lo:hi] = (s * delta).max(axis=2).sum(axis=0) / V
    return S


def fif_scores_lists(Q, q_off, q_codes, X, lists):
    """Eq. 4 evaluated through the first inverted file, float64 [B, N].

    For each query view q_i, only the lists of its codewords are visited; per
    shape the max over the visited entries is taken, and 0 joins that max when
    some view of the shape was not visited (those products are 0 in Eq. 4).
    Shapes never visited score 0 for q_i. A view reached through several lists
    (multiple assignment on both sides) counts once.
    """
    X = np.asarray(X)
    N, Nv, D = X.shape
    q_codes = np.asarray(q_codes)
    q_off = np.asarray(q_off)
    B = len(q_off) - 1
    S = np.zeros((B, N))
    for b in range(B):
        V = q_off[b + 1] - q_off[b]
        for i in range(q_off[b], q_off[b + 1]):
            best = {}
            seen = {}
            for c in q_codes[i]:
                ent = lists[int(c)]
                if len(ent) == 0:
                    continue
                s = cosine(Q[i:i + 1], X[ent[:, 0], ent[:, 1]])[0]
                for (p, j), v in zip(ent, s):
                    p = int(p)
                    best[p] = max(best.get(p, -np.inf), v)
                    seen.setdefault(p, set()).add(int(j))
            for p, v in best.items():
                if len(seen[p]) < Nv:
                    v = max(v, 0.0)
                S[b, p] += v / V
    return S


def fif_upper_bound(Q, q_off, views_of, n_shapes, chunk_shapes=1024):
    """U(x_q, x_p) = (1/|V(x_q)|) sum_i max(0, max_j s(q_i, p_j)), float64 [B, N].

    Every term of Eq. 4 is at most max(0, max_j s(q_i, p_j)): the delta keeps a
    subset of the products and contributes 0 for the rest. So U bounds the
    Eq. 4 score from above (it equals Eq. 3 when all cosines are >= 0).
    ``views_of(first, n)`` returns the views [n, N_v, D] of database shapes
    [first, first + n); the next chunk is drawn while the current one is used.
    """
    from concurrent.futures import ThreadPoolExecutor
    q_off = np.asarray(q_off)
    B = len(q_off) - 1
    U = np.zeros((B, n_shapes))
    Qa = _f64(Q[:q_off[-1]])
    starts = list(range(0, n_shapes, chunk_shapes))
    with ThreadPoolExecutor(1) as ex:
        nxt = ex.submit(views_of, 0, min(chunk_shapes, n_shapes)) if starts else None
        for c, lo in enumerate(starts):
            X = np.asarray(nxt.result())
            n, Nv, D = X.shape
            if c + 1 < len(starts):
                lo2 = starts[c + 1]
                nxt = ex.submit(views_of, lo2, min(chunk_shapes, n_shapes - lo2))
            s = cosine(Qa, X.reshape(n * Nv, D)).reshape(-1, n, Nv)
            m = np.maximum(s.max(axis=2), 0.0)
            for b in range(B):
                U[b, lo:lo + n] = m[q_off[b]:q_off[b + 1]].sum(axis=0) / (q_off[b + 1] - q_off[b])
    return U


def fif_topk_bounded(Q, q_off, q_codes, codebook, views_of_shape, U, k, group=128, views_of_group=None):
    """Top-k of Eq. 4 for each query, quantising only the shapes it must visit.

    Shapes are visited in order of the upper bound U (``fif_upper_bound``,
    desc, ties by id); the views of each visited shape are quantised
    (``quantize``, one assignment) and its Eq. 4 score computed
    (``fif_scores``). The walk stops once k shapes are scored and the k-th
    best score exceeds the bound of the next shape: no shape left can enter
    the top-k. ``views_of_shape(p)`` returns the views [N_v, D] of shape p
    (``views_of_group(ids)``, if given, those of several shapes at once).
    Returns ([(ids, scores)] ordered by (score desc, id asc) per query, the
    number of shapes visited per query).
    """
    q_off = np.asarray(q_off)
    q_codes = np.asarray(q_codes)
    B, N = U.shape
    codes_cache = {}
    out, visited = [], []
    for b in range(B):
        order = np.lexsort((np.arange(N), -U[b]))
        Qb = Q[q_off[b]:q_off[b + 1]]
        cb = q_codes[q_off[b]:q_off[b + 1]]
        found_ids, found_sc = [], []
        pos = 0
        while pos < N:
            ids = order[pos:pos + group]
            Xg = views_of_group(ids) if views_of_group else np.stack([views_of_shape(int(p)) for p in ids])
            need = [i for i, p in enumerate(ids) if int(p) not in codes_cache]
            if need:
                cg = quantize(Xg[need].reshape(-1, Xg.shape[2]), codebook, 1).reshape(len(need), -1)
                for r, i in enumerate(need):
                    codes_cache[int(ids[i])] = cg[r]
            dbc = np.stack([codes_cache[int(p)] for p in ids])
            sc = fif_scores(Qb, np.array([0, len(Qb)]), cb, Xg, dbc)[0]
            found_ids.extend(int(p) for p in ids)
            found_sc.extend(sc.tolist())
            pos += len(ids)
            if len(found_sc) >= k and pos < N:
                kth = np.sort(np.asarray(found_sc))[::-1][k - 1]
                if kth > U[b, order[pos]]:
                    break
        fi = np.asarray(found_ids, np.int64)
        fs = np.asarray(found_sc)
        o = np.lexsort((fi, -fs))[:k]
        out.append((fi[o], fs[o]))
        visited.append(pos)
    return out, visited


def rank(scores, k):
    """Top-k of one score row: (ids int64 [k], scores [k]) ordered by (score desc, id asc)."""
    s = _f64(scores)
    order = np.lexsort((np.arange(s.shape[0]), -s))[:k]
    return order, s[order]


def membership(scores, k1):
    """Sparse activation F_q of Eq. 7: F[i] = S(x_q, x_i) if x_i in N_k1(x_q) else 0.

    N_k1 is the first k1 entries of the ranking of ``scores`` (float64 [N]).
    F is a fuzzy-set membership (Eq. 8 compares memberships by min and max), so a
    neighbour whose score is negative -- possible only with signed features --
    has membership 0.
    """
    ids, vals = rank(scores, k1)
    F = np.zeros(np.asarray(scores).shape[0])
    F[ids] = np.maximum(vals, 0.0)
    return F


def contextual(Fq, Fp):
    """Eq. 8: S'(x_q, x_p) = sum_i min(F_q[i], F_p[i]) / sum_i max(F_q[i], F_p[i]).

    Returns 0 when the denominator is 0 (both vectors zero).
    """
    Fq = _f64(Fq)
    Fp = _f64(Fp)
    den = np.maximum(Fq, Fp).sum()
    if den == 0:
        return 0.0
    return float(np.minimum(Fq, Fp).sum() / den)


def db_memberships(S_db, k1):
    """Dense F_p for every database shape p (rows of float64 [N, N]).

    ``S_db[p]`` is the score row of shape p used as a query (self included).
    """
    S_db = _f64(S_db)
    return np.stack([membership(S_db[p], k1) for p in range(S_db.shape[0])])


def build_sif(F_db):
    """Second inverted file (Fig. 3): N entries; entry i stores ||F_i||_1 and the
    pairs (p, F_p[i]) of every shape p whose activation at i is non-zero, p ascending.

    Returns (card float64 [N], entries: list of (ids int64, values float64)).
    """
    F_db = _f64(F_db)
    N = F_db.shape[0]
    card = F_db.sum(axis=1)
    entries = []
    for i in range(N):
        ps = np.nonzero(F_db[:, i])[0]
        entries.append((ps.astype(np.int64), F_db[ps, i]))
    return card, entries


def sif_scores_inverted(Fq, card, entries):
    """S'(x_q, .) over all N shapes through the second inverted file.

    Numerator, Eq. 13: sum over i with F_q[i] != 0 and F_p[i] != 0 of
    min(F_q[i], F_p[i]), gathered by walking entry i for each non-zero F_q[i].
    Denominator, Eq. 14: ||F_q||_1 + ||F_p||_1 - numerator.
    """
    Fq = _f64(Fq)
    N = Fq.shape[0]
    num = np.zeros(N)
    for i in np.nonzero(Fq)[0]:
        ps, vals = entries[i]
        for p, v in zip(ps, vals):
            num[p] += min(Fq[i], v)
    den = Fq.sum() + card - num
    out = np.zeros(N)
    nz = den > 0
    out[nz] = num[nz] / den[nz]
    return out


def rerank(S_q, F_db, k1, k):
    """Re-ranked top-k of each query, ordered by (S' desc, S desc, id asc).

    S' (Eq. 8) is computed densely over all N shapes from F_q (Eq. 7, built from
    the query's first k1 neighbours) and the database rows F_db.
    Returns (ids int64 [B, k], S' float64 [B, k]).
    """
    S_q = np.atleast_2d(_f64(S_q))
    B, N = S_q.shape
    ids = np.zeros((B, k), np.int64)
    sp = np.zeros((B, k))
    for b in range(B):
        Fq = membership(S_q[b], k1)
        Sprime = np.array([contextual(Fq, F_db[p]) for p in range(N)])
        order = np.lexsort((np.arange(N), -S_q[b], -Sprime))[:k]
        ids[b] = order
        sp[b] = Sprime[order]
    return ids, sp


def augment(F_rows, nbrs):
    """Eq. 10 (and each line of Eq. 11): the mean of the activations F_i of the
    shapes i in the neighbour set ``nbrs`` (ids); ``F_rows`` float64 [N, N]."""
    nbrs = np.asarray(nbrs, np.int64)
    return _f64(F_rows)[nbrs].sum(axis=0) / len(nbrs)


def aca_fuse(F1, F2, alpha):
    """Eq. 9: element-wise generalised mean with exponent alpha of two activations."""
    F1 = _f64(F1)
    F2 = _f64(F2)
    return ((F1 ** alpha + F2 ** alpha) / 2.0) ** (1.0 / alpha)


def aca_activation(S1, S2, F1_db, F2_db, k1, k2, alpha, mode):
    """Aggregated contextual activation (Sec. 2.4) of one shape from its two score rows.

    mode "none": F^(l) = Eq. 7 of measure l (first k1 neighbours);
    mode "aug":  F^(l) = Eq. 10, the mean of the database activations F_i^(l)
                 over the shape's first k2 neighbours under measure l;
    mode "co":   Eq. 11, the same mean over the first k2 neighbours under the
                 other measure;
    then Eq. 9 fuses F^(1) and F^(2). ``F1_db``/``F2_db`` are the database
    activations (Eq. 7 rows, ``db_memberships``).
    """
    if mode == "none":
        A1, A2 = membership(S1, k1), membership(S2, k1)
    else:
        n1 = rank(S1, k2)[0]
        n2 = rank(S2, k2)[0]
        if mode == "aug":
            A1, A2 = augment(F1_db, n1), augment(F2_db, n2)
        elif mode == "co":
            A1, A2 = augment(F1_db, n2), augment(F2_db, n1)
        else:
            raise ValueError(mode)
    return aca_fuse(A1, A2, alpha)


def aca_db(S1_db, S2_db, k1, k2, alpha, mode):
    """ACA rows of every database shape, float64 [N, N]; row p uses the score
    rows of p matched as a query under each measure (self included)."""
    F1_db, F2_db = db_memberships(S1_db, k1), db_memberships(S2_db, k1)
    N = F1_db.shape[0]
    return np.stack([aca_activation(S1_db[p], S2_db[p], F1_db, F2_db, k1, k2, alpha, mode) for p in range(N)])


def rerank_aca(S1_q, S2_q, S1_db, S2_db, k1, k2, alpha, mode, k):
    """Re-ranked top-k with two similarity measures (the paper's default re-ranking):
    ACA of the query and of every database shape (``aca_activation``), S' of
    Eq. 8 between them over all N shapes, order (S' desc, S^(1) desc, id asc).
    Returns (ids int64 [B, k], S' float64 [B, k])."""
    S1_q = np.atleast_2d(_f64(S1_q))
    S2_q = np.atleast_2d(_f64(S2_q))
    F1_db, F2_db = db_memberships(S1_db, k1), db_memberships(S2_db, k1)
    A_db = aca_db(S1_db, S2_db, k1, k2, alpha, mode)
    B, N = S1_q.shape
    ids = np.zeros((B, k), np.int64)
    sp = np.zeros((B, k))
    for b in range(B):
        Fq = aca_activation(S1_q[b], S2_q[b], F1_db, F2_db, k1, k2, alpha, mode)
        Sprime = np.array([contextual(Fq, A_db[p]) for p in range(N)])
        order = np.lexsort((np.arange(N), -S1_q[b], -Sprime))[:k]
        ids[b] = order
        sp[b] = Sprime[order]
    return ids, sp


# ---------------------------------------------------------------- projection rendering (Sec. 2.1)
def normalize_mesh(V, T):
    """Scale and translation normalisation of Sec. 2.1: the centroid of the surface
    (triangle centroids weighted by area) goes to the origin and the largest
    distance of a surface point from it becomes 1. Returns (centre [3], scale)."""
    V = _f64(V)
    T = np.asarray(T, np.int64)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    centre = (area[:, None] * (a + b + c) / 3.0).sum(axis=0) / area.sum()
    return centre, 1.0 / np.sqrt(((V - centre) ** 2).sum(axis=1)).max()


def view_frames(n_az, n_el):
    """Cameras on the unit sphere at azimuth 2 pi i / n_az and elevation
    pi ((j + 1/2) / n_el - 1/2), view v = j * n_az + i, each looking at the origin:
    (position C, forward f = -C, right r = f x z / |f x z|, up u = r x f), [N_v, 3] each."""
    az = 2 * np.pi * np.arange(n_az) / n_az
    el = np.pi * ((np.arange(n_el) + 0.5) / n_el - 0.5)
    E, A = np.meshgrid(el, az, indexing="ij")
    C = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1).reshape(-1, 3)
    f = -C
    r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    u = np.cross(r, f)
    return C, f, r, u


def raster_depth(S, T, H, W, background=2.0):
    """Depth buffer of triangles given in screen space S [n, 3] = (x, y, depth), x and y
    in [-1, 1]: pixel (i, j) samples its centre (-1 + (2j + 1)/W, 1 - (2i + 1)/H); a
    sample is covered when all three edge functions of the triangle, oriented to a
    positive area, are >= 0 (degenerate triangles cover nothing); its depth is the
    barycentric interpolation, and the nearest (smallest) depth is kept."""
    S = _f64(S)
    T = np.asarray(T, np.int64)
    D = np.full((H, W), float(background))
    xs = -1 + (2 * np.arange(W) + 1) / W
    ys = 1 - (2 * np.arange(H) + 1) / H
    for t in T:
        a, b, c = S[t[0]], S[t[1]], S[t[2]]
        area = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        if area == 0:
            continue
        if area < 0:
            b, c = c, b
            area = -area
        jj = np.nonzero((xs >= min(a[0], b[0], c[0])) & (xs <= max(a[0], b[0], c[0])))[0]
        ii = np.nonzero((ys >= min(a[1], b[1], c[1])) & (ys <= max(a[1], b[1], c[1])))[0]
        if len(jj) == 0 or len(ii) == 0:
            continue
        X, Y = np.meshgrid(xs[jj], ys[ii])
        ea = (c[0] - b[0]) * (Y - b[1]) - (c[1] - b[1]) * (X - b[0])  # opposite a
        eb = (a[0] - c[0]) * (Y - c[1]) - (a[1] - c[1]) * (X - c[0])  # opposite b
        ec = (b[0] - a[0]) * (Y - a[1]) - (b[1] - a[1]) * (X - a[0])  # opposite c
        inside = (ea >= 0) & (eb >= 0) & (ec >= 0)
        z = (ea * a[2] + eb * b[2] + ec * c[2]) / area
        sub = D[np.ix_(ii, jj)]
        D[np.ix_(ii, jj)] = np.where(inside, np.minimum(sub, z), sub)
    return D


def render_depth(V, T, n_az, n_el, H, W):
    """The N_v = n_az * n_el depth views of Sec. 2.1 of one mesh, float64 [N_v, H, W]:
    normalise (``normalize_mesh``), then for every camera of ``view_frames`` an
    orthographic depth buffer along its forward axis, depth = distance from the
    camera's tangent plane, p . f + 1 in [0, 2] (2 where nothing is seen)."""
    centre, scale = normalize_mesh(V, T)
    P = (_f64(V) - centre) * scale
    _, f, r, u = view_frames(n_az, n_el)
    out = np.empty((len(f), H, W))
    for v in range(len(f)):
        S = np.stack([P @ r[v], P @ u[v], P @ f[v] + 1.0], axis=1)
        out[v] = raster_depth(S, T, H, W)
    return out


def match_forward(Q, q_off, P, W=None):
    """Eq. 3 after a linear view projection u = W q, v = W p.

    Returns (S float64 [B, Np], jstar int64 [sum V_q, Np]) where jstar[i, p] is
    the first j attaining max_j s(u_i, v_j) (lowest index on ties).
    """
    Q = _f64(Q)
    P = _f64(P)
    Np, nv, din = P.shape
    Wm = np.eye(din) if W is None else _f64(W)
    U = Q @ Wm.T
    V = P.reshape(Np * nv, din) @ Wm.T
    q_off = np.asarray(q_off)
    B = len(q_off) - 1
    S = np.zeros((B, Np))
    jstar = np.zeros((Q.shape[0], Np), np.int64)
    for b in range(B):
        lo, hi = q_off[b], q_off[b + 1]
        s = cosine(U[lo:hi], V).reshape(hi - lo, Np, nv)
        jstar[lo:hi] = s.argmax(axis=2)
        S[b] = s.max(axis=2).sum(axis=0) / (hi - lo)
    return S, jstar


def match_backward(Q, q_off, P, W, G):
    """Gradient of L = sum_{b,p} G[b,p] S(x_b, x_p) through ``match_forward``.

    With u_i = W q_i, v_j = W p_j and s_ij = u_i.v_j / (|u_i||v_j|), the max of
    Eq. 3 picks j* per (i, p), and
      dS/du_i     = (v_j*/|v_j*| - s u_i/|u_i|) / |u_i|,
      dS/dv_j*    = (u_i/|u_i|  - s v_j*/|v_j*|) / |v_j*|,
    each scaled by G[b, p] / |V(x_b)|; then dW = sum dU q^T + sum dV p^T,
    dQ = dU W, dP = dV W (W = identity when None).
    Returns (dW or None, dQ [sum V_q, din], dP [Np, nv, din]).
    """
    Q = _f64(Q)
    P = _f64(P)
    G = _f64(G)
    Np, nv, din = P.shape
    Wm = np.eye(din) if W is None else _f64(W)
    U = Q @ Wm.T
    V = P.reshape(Np * nv, din) @ Wm.T
    nu = np.linalg.norm(U, axis=1)
    nvv = np.linalg.norm(V, axis=1)
    dU = np.zeros_like(U)
    dV = np.zeros_like(V)
    q_off = np.asarray(q_off)
    B = len(q_off) - 1
    for b in range(B):
        lo, hi = q_off[b], q_off[b + 1]
        Vb = hi - lo
        for i in range(lo, hi):
            ui = U[i] / nu[i]
            for p in range(Np):
                blk = V[p * nv:(p + 1) * nv]
                s = blk @ ui / nvv[p * nv:(p + 1) * nv]
                j = int(np.argmax(s))
                r = p * nv + j
                vj = V[r] / nvv[r]
                c = G[b, p] / Vb
                dU[i] += c * (vj - s[j] * ui) / nu[i]
                dV[r] += c * (ui - s[j] * vj) / nvv[r]
    dQ = dU @ Wm
    dP = (dV @ Wm).reshape(Np, nv, din)
    dW = None if W is None else dU.T @ Q + dV.T @ P.reshape(Np * nv, din)
    return dW, dQ, dP
