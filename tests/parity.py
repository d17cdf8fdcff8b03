"""Comparison rules between the CUDA path and the FP64 oracle.

* codes: identical wherever the oracle's own margin between the codewords that
  decide them exceeds MARGIN * ||x||^2; rows under that margin are counted.
* scores: |gpu - oracle| <= RTOL * |oracle| + ATOL (FP32 paths).
* top-k ids: every returned score is the oracle's score of that id (within the
  score tolerance); the j-th returned score matches the oracle's j-th best; ids
  are identical at every rank whose oracle score is separated from its
  neighbours by more than the tolerance (several orders are correct there).
"""
import numpy as np

from oracle import gift_oracle as O

MARGIN = 1e-6
RTOL = 1e-5
ATOL = 1e-6


def code_margins(X, codebook, ma):
    """FP64 margin of each row: min gap among the first ma+1 sorted distances, / ||x||^2."""
    X = np.asarray(X, np.float64)
    d = np.sort(O.sq_distances(X, codebook), axis=1)[:, :ma + 1]
    gaps = np.diff(d, axis=1).min(axis=1) if d.shape[1] > 1 else np.full(len(X), np.inf)
    xx = np.maximum((X * X).sum(1), 1e-300)
    return gaps / xx


def assert_codes(gpu_codes, ref_codes, margins, max_untied_mismatch=0):
    gpu_codes = np.asarray(gpu_codes).reshape(ref_codes.shape)
    bad = np.any(gpu_codes != ref_codes, axis=1)
    tied = margins <= MARGIN
    assert np.sum(bad & ~tied) <= max_untied_mismatch, (
        f"{np.sum(bad & ~tied)} codes differ above the margin; first rows {np.nonzero(bad & ~tied)[0][:8]}")
    return int(np.sum(bad)), int(np.sum(tied))


def close(a, b, rtol=RTOL, atol=ATOL):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) <= rtol * np.abs(b) + atol


def assert_topk(gpu_ids, gpu_scores, ref_row, k, rtol=RTOL, atol=ATOL):
    """GPU top-k of one query against the oracle's full FP64 score row."""
    gpu_ids = np.asarray(gpu_ids, np.int64)
    gpu_scores = np.asarray(gpu_scores, np.float64)
    ref_ids, ref_sc = O.rank(ref_row, k)
    assert len(set(gpu_ids.tolist())) == len(gpu_ids), "duplicate ids"
    ok = close(gpu_scores, ref_row[gpu_ids], rtol, atol)
    assert ok.all(), f"scores of returned ids differ: {np.nonzero(~ok)[0][:5]}"
    ok = close(gpu_scores, ref_sc, rtol, atol)
    assert ok.all(), f"ranked scores differ at ranks {np.nonzero(~ok)[0][:5]}"
    # ranks whose oracle score is isolated from both neighbours must match exactly
    full = np.sort(np.asarray(ref_row, np.float64))[::-1][:k + 1]
    tol = rtol * np.abs(full) + atol
    for j in range(k):
        lo_gap = full[j] - full[j + 1] if j + 1 < len(full) else np.inf
        hi_gap = full[j - 1] - full[j] if j > 0 else np.inf
        if lo_gap > 2 * tol[j] and hi_gap > 2 * tol[j]:
            assert gpu_ids[j] == ref_ids[j], f"rank {j}: gpu {gpu_ids[j]} oracle {ref_ids[j]}"


def recall(gpu_ids, ref_row, k):
    ref_ids, _ = O.rank(ref_row, k)
    return len(set(np.asarray(gpu_ids[:k]).tolist()) & set(ref_ids.tolist())) / k


# ---------------------------------------------------------------- S' (Eq. 8)
# Memberships on the GPU are FP32 scores, F' = F (1 + eta) + zeta: a relative
# error eta inside a band [L, H] (L <= 0 <= H), and an additive part zeta --
# the fixed-point rounding of round(F' 2^31) (at most 2^-32) plus, for
# memberships near 0, an absolute score error a. min and max are monotone, so
# the min (max) of two memberships with relative errors in [L, H] lies in
# [(1 + L), (1 + H)] times the exact min (max): the exact integer sums of
# Eq. 13 (k1 terms) and Eq. 14 (at most 2 k1 terms) stay in that band up to
# 2^-32 + a per term, and S' = num / den moves by at most (H - L) / (1 + L)
# relative (a bias shared by all memberships cancels), plus three FP32
# roundings of 2^-24 in its conversions and division. With den >= ||F_q||_1:
#   |S'_gpu - S'| <= ((H - L) / (1 + L) + 4 * 2^-24) S' + 3 k1 (2^-32 + a) / ||F_q||_1.
FIX = 2.0 ** -31  # membership fixed point


class ErrorBand:
    """Band [L, H] of the GPU memberships' relative errors against the oracle's, and
    the largest absolute error a of memberships at or below a floor."""

    def __init__(self):
        self.lo, self.hi, self.abs = 0.0, 0.0, 0.0

    def add(self, gpu, ref, floor=0.0):
        gpu = np.asarray(gpu, np.float64)
        ref = np.asarray(ref, np.float64)
        d = gpu - ref
        d = np.sign(d) * np.maximum(np.abs(d) - FIX / 2, 0.0)  # fixed-point rounding is counted apart
        big = ref > floor
        if big.any():
            r = d[big] / ref[big]
            self.lo, self.hi = min(self.lo, float(r.min())), max(self.hi, float(r.max()))
        small = ~big & ((ref != 0) | (gpu != 0))
        if small.any():
            self.abs = max(self.abs, float(np.abs(d[small]).max()))
        return self

    def sprime_tolerance(self, k1, fq_norm):
        """(rtol, atol) of S' from the bound above."""
        rtol = (self.hi - self.lo) / (1.0 + self.lo) + 4 * 2.0 ** -24
        return rtol, 3 * k1 * (2.0 ** -32 + self.abs) / max(float(fq_norm), 1e-30)


def sif_rows(off, ids, mem, N):
    """Dense [N, N] memberships F_p[i] from an exported S-IF (entry i lists (p, F_p[i]))."""
    F = np.zeros((N, N))
    for i in range(N):
        F[ids[off[i]:off[i + 1]], i] = mem[off[i]:off[i + 1]] * FIX
    return F


def sif_sets(off, ids, N):
    """Neighbour sets N_k1(p) of an exported S-IF as a bool [N, N] matrix (p, i):
    entry i lists p for every i in N_k1(p), zero memberships included."""
    M = np.zeros((N, N), bool)
    for i in range(N):
        M[ids[off[i]:off[i + 1]], i] = True
    return M


def reference_memberships(ref_row, gpu_set, k1, rtol=RTOL, atol=ATOL):
    """The oracle's Eq. 7 memberships on the GPU's neighbour set, after checking that
    the set is a correct first-k1 set of the oracle's ranking: k1 members, each with
    an oracle score within the score tolerance of the oracle's k1-th score (near ties
    at the k1 boundary admit several correct sets)."""
    ref_row = np.asarray(ref_row, np.float64)
    gpu_set = np.asarray(gpu_set, np.int64)
    k = min(k1, len(ref_row))
    assert len(set(gpu_set.tolist())) == len(gpu_set) == k, "neighbour set size"
    kth = np.sort(ref_row)[::-1][k - 1]
    assert np.all(ref_row[gpu_set] >= kth - 2 * (rtol * abs(kth) + atol)), "neighbour set is not a first-k1 set"
    F = np.zeros(len(ref_row))
    F[gpu_set] = np.maximum(ref_row[gpu_set], 0.0)
    return F
