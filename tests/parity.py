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
