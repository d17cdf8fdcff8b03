"""Serving loop: each request's result is the same alone and inside a mix of
concurrent requests with mixed view counts; bounded waits report a timeout."""
import threading
import time

import numpy as np
import pytest

from synth import shape_views, query_views, kmeans_codebook

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(gpu_lib):
    import torch
    N, Nv, D, C, K = 300, 64, 128, 15, 24
    X = shape_views(0, N, Nv, D, C, 1401, 4401)
    cb = kmeans_codebook(X.reshape(-1, D), K, 3401, 8)
    ix = gpu_lib.Index(torch.from_numpy(X).cuda(), torch.from_numpy(cb).cuda(), N, Nv, K, storage="bf16",
                       rescore_r=40, sif_k1=10, keep_exact=False)
    Q, qoff, _ = query_views(60, (12, 20, 64), D, C, 2401, 4401, max_views=64)
    queries = [Q[qoff[b]:qoff[b + 1]] for b in range(len(qoff) - 1)]
    yield gpu_lib, ix, queries
    ix.close()


def test_same_result_alone_and_in_a_mix(served):
    gift, ix, queries = served
    sv = gift.Server(ix, slots=3, max_batch_queries=16, max_batch_views=16 * 64, topk=20, rerank=True)
    try:
        alone = []
        for q in queries:
            alone.append(sv.wait(sv.submit(q)))
        assert sv.stats()["mean_batch"] == pytest.approx(1.0)
        tickets = [None] * len(queries)
        g = np.random.default_rng(7)
        gaps = g.exponential(1.0 / 4000.0, size=len(queries))  # Poisson arrivals, 4,000 requests/s

        def producer():
            t = time.perf_counter()
            for i, q in enumerate(queries):
                t += gaps[i]
                while time.perf_counter() < t:
                    pass
                tickets[i] = sv.submit(q)

        th = threading.Thread(target=producer)
        th.start()
        th.join()
        mixed = [sv.wait(t) for t in tickets]
        st = sv.stats()
        assert st["completed"] == 2 * len(queries) and st["failed"] == 0
        assert st["batches"] < 2 * len(queries)  # requests were batched together
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        for (ia, sa), (ib, sb) in zip(alone, mixed):
            assert np.array_equal(ia, ib)
            assert np.allclose(sa, sb, rtol=1e-5, atol=1e-6)
    finally:
        sv.close()


def test_served_results_equal_direct_calls(served):
    import torch
    gift, ix, queries = served
    sv = gift.Server(ix, slots=2, max_batch_queries=8, max_batch_views=8 * 64, topk=20, rerank=False)
    try:
        q = queries[:5]
        got = [sv.wait(sv.submit(x)) for x in q]
    finally:
        sv.close()
    off = np.concatenate([[0], np.cumsum([len(x) for x in q])]).astype(np.int32)
    ids, sc = ix.query(torch.from_numpy(np.concatenate(q)).cuda(), off, mode="fif", topk=20)
    for b in range(5):
        assert np.array_equal(got[b][0], ids[b].cpu().numpy())
        assert np.allclose(got[b][1], sc[b].cpu().numpy(), rtol=1e-6, atol=1e-7)


def test_bounded_wait_times_out_and_recovers(served):
    gift, ix, queries = served
    sv = gift.Server(ix, slots=1, max_batch_queries=4, max_batch_views=4 * 64, topk=10, rerank=True,
                     start_paused=True)
    try:
        t = sv.submit(queries[0])
        with pytest.raises(gift.GiftError) as e:
            sv.wait(t, timeout_ms=50)
        assert e.value.status == 4  # GIFT_ETIMEOUT
        sv.resume()
        ids, sc = sv.wait(t, timeout_ms=60000)
        assert ids.shape == (10,) and np.all(ids >= 0)
        with pytest.raises(gift.GiftError):
            sv.wait(t, timeout_ms=10)  # ticket already consumed
        with pytest.raises(gift.GiftError):
            sv.submit(np.zeros((4 * 64 + 1, ix.dim), np.float32))  # more views than a batch holds
    finally:
        sv.close()


def test_memory_admission_holds_batches_back(served):
    """A memory budget that fits one full batch in flight: the dispatcher must hold later
    batches back until memory frees up (admission_waits > 0, the admitted bytes never above
    the budget while more than one batch is in flight), and every result still equals the
    request's result alone."""
    gift, ix, queries = served
    kw = dict(slots=3, max_batch_queries=16, max_batch_views=16 * 64, topk=20, rerank=True)
    probe = gift.Server(ix, **kw)
    st0 = probe.stats()
    alone = [probe.wait(probe.submit(q)) for q in queries]
    probe.close()
    budget = st0["slot_bytes"] + st0["max_batch_bytes"] * 3 // 2  # one full batch, not two
    sv = gift.Server(ix, memory_budget=budget, start_paused=True, **kw)
    try:
        tickets = [sv.submit(q) for q in queries * 3]  # queued while paused: full batches from the start
        sv.resume()
        mixed = [sv.wait(t) for t in tickets]
        st = sv.stats()
        assert st["budget_bytes"] == budget - st0["slot_bytes"]
        assert st["admission_waits"] > 0, st
        assert st["peak_in_flight_bytes"] <= max(st["budget_bytes"], st["max_batch_bytes"]), st
        assert st["completed"] == 3 * len(queries) and st["failed"] == 0
        for k, (ib, sb) in enumerate(mixed):
            ia, sa = alone[k % len(queries)]
            assert np.array_equal(ia, ib)
            assert np.allclose(sa, sb, rtol=1e-5, atol=1e-6)
    finally:
        sv.close()
