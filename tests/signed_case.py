"""Signed-feature cases shared by the CPU check of the fixture and the GPU parity
tests: cosines take both signs, so Eq. 4's per-(query view, shape) maximum can be
negative. It stays negative only when every view of the shape shares a codeword
with the query view; otherwise the 0 of an unmatched view joins the max."""
import numpy as np

from oracle import gift_oracle as O
from synth import kmeans_codebook, signed_views

# pure-noise views, 3 per shape, K = 3: lists of ~300 entries (several scan tiles)
SIGNED = dict(N=300, Nv=3, D=128, C=4, K=3)


def signed_case(ma=1, db_ma=1, seed=21, nq=8, qviews=(8, 5, 3), **kw):
    """(X [N, Nv, D], codebook [K, D], Q [sum V_q, D], q_off [B+1], db codes [N, Nv, db_ma], query codes)."""
    c = dict(SIGNED, **kw)
    N, Nv, D, C, K = c["N"], c["Nv"], c["D"], c["C"], c["K"]
    X = signed_views(N, Nv, D, C, 1000 + seed, 4000 + seed, weight=0.0)
    cb = kmeans_codebook(X.reshape(-1, D), K, 3000 + seed, 8) if K > 1 else np.ones((1, D), np.float32)
    full = signed_views(nq, max(qviews), D, C, 2000 + seed, 4000 + seed, weight=0.0)
    counts = [qviews[b % len(qviews)] for b in range(nq)]
    Q = np.concatenate([full[b, :counts[b]] for b in range(nq)])
    q_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    dbc = O.quantize(X.reshape(-1, D), cb, db_ma).reshape(N, Nv, db_ma)
    return X, cb, Q, q_off, dbc, O.quantize(Q, cb, ma)


def negative_terms(X, Q, dbc, qc):
    """Counts of (query view, shape) pairs reached through a list whose matched
    views all have negative cosines: (all views of the shape matched, some not)."""
    N, Nv, D = X.shape
    s = O.cosine(Q, X.reshape(-1, D)).reshape(len(Q), N, Nv)
    delta = (dbc[None, :, :, :, None] == qc[:, None, None, None, :]).any(axis=(3, 4))
    neg = np.where(delta, s, -np.inf).max(axis=2) < 0
    covered = delta.all(axis=2)
    return int((neg & covered).sum()), int((neg & ~covered & delta.any(axis=2)).sum())
