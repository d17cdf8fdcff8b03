"""Streamed (three-pass, chunked) index build against the one-shot build.

Both builds run the same kernels on the same rows, so the F-IF lists, the
S-IF and the query results must be identical; the oracle pins the streamed
index's top-k as well. Chunks come in uneven sizes, out of order, and from
host and device memory.
"""
import ctypes

import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import shape_views, query_views, kmeans_codebook
from tests.parity import assert_topk

pytestmark = pytest.mark.gpu

N, NV, D, C, K = 200, 64, 128, 20, 64


@pytest.fixture(scope="module")
def data():
    X = shape_views(0, N, NV, D, C, 1101, 4101)
    cb = kmeans_codebook(X.reshape(-1, D), K, 3101, 8)
    Q, qoff, _ = query_views(12, (64, 17, 40), D, C, 2101, 4101, max_views=64)
    return X, cb, Q, qoff


def _chunks(n_shapes, sizes):
    out, f, i = [], 0, 0
    while f < n_shapes:
        n = min(sizes[i % len(sizes)], n_shapes - f)
        out.append((f, n))
        f += n
        i += 1
    return out


def _streamed(gift, torch, X, cb, storage, rescore_r, sif_k1, order_seed=0):
    lib = gift.load()
    prm = gift._Params(N, NV, D, K, gift._STORAGE[storage], 1, sif_k1, rescore_r, 0)
    h = ctypes.c_void_p()
    st = gift._stream()
    gift._check(lib.gift_build_begin(ctypes.byref(prm), gift._ptr(torch.from_numpy(cb).cuda()), st, ctypes.byref(h)))
    ix = gift.Index.__new__(gift.Index)
    ix._h, ix.params = h, prm
    ix.n_shapes, ix.views_per_shape, ix.dim, ix.n_codewords = N, NV, D, K
    ix.query_ma, ix.sif_k1, ix.rescore_r = 1, sif_k1, rescore_r
    g = np.random.default_rng(order_seed)
    for p in (1, 2, 3):
        if p == 3 and sif_k1 == 0:
            break
        ch = _chunks(N, [37, 1, 64, 23])
        g.shuffle(ch)
        for j, (f, n) in enumerate(ch):
            x = np.ascontiguousarray(X[f:f + n])
            buf = x if (j + p) % 2 else torch.from_numpy(x).cuda()  # host and device chunks
            gift._check(lib.gift_build_add(h, p, gift._ptr(buf), f, n, st))
        gift._check(lib.gift_build_end_pass(h, p, st))
    return ix


@pytest.mark.parametrize("storage,rescore_r,sif_k1", [("bf16", 40, 10), ("fp8", 40, 10), ("f32", 0, 0),
                                                      ("bf16", 0, 12)])
def test_streamed_equals_one_shot(gpu_lib, data, storage, rescore_r, sif_k1):
    import torch
    X, cb, Q, qoff = data
    one = gpu_lib.Index(torch.from_numpy(X).cuda(), torch.from_numpy(cb).cuda(), N, NV, K, storage=storage,
                        sif_k1=sif_k1, rescore_r=rescore_r, keep_exact=False)
    st = _streamed(gpu_lib, torch, X, cb, storage, rescore_r, sif_k1)
    for a, b in zip(one.export_fif(), st.export_fif()):
        assert np.array_equal(a, b)
    if sif_k1:
        for a, b in zip(one.export_sif(), st.export_sif()):
            assert np.array_equal(a, b)
    q = torch.from_numpy(Q).cuda()
    k = 10
    i1, s1 = one.query(q, qoff, topk=k)
    i2, s2 = st.query(q, qoff, topk=k)
    assert torch.equal(i1, i2) and torch.equal(s1, s2)
    if sif_k1:
        r1 = one.rerank(i1, s1, k1=min(sif_k1, k), topk=5)
        r2 = st.rerank(i2, s2, k1=min(sif_k1, k), topk=5)
        assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1])
    # the streamed index against the oracle's Eq. 4 ranking (FP32-level scores only)
    if storage == "f32" or rescore_r:
        dbc = O.quantize(X.reshape(-1, D), cb, 1).reshape(N, NV)
        ref = O.fif_scores(Q, np.asarray(qoff), O.quantize(Q, cb, 1), X, dbc)
        ids, sc = i2.cpu().numpy(), s2.cpu().numpy()
        for b in range(len(qoff) - 1):
            assert_topk(ids[b], sc[b], ref[b], k)
    one.close()
    st.close()


def test_binding_builds_from_a_generator(gpu_lib, data):
    import torch
    X, cb, Q, qoff = data
    calls = []

    def chunk(f, n):
        calls.append((f, n))
        return shape_views(0, N, NV, D, C, 1101, 4101)[f:f + n]

    st = gpu_lib.Index.streamed(chunk, torch.from_numpy(cb).cuda(), N, NV, K, chunk_shapes=48, storage="bf16",
                                sif_k1=8, rescore_r=20)
    assert len(calls) == 3 * 5
    one = gpu_lib.Index(torch.from_numpy(X).cuda(), torch.from_numpy(cb).cuda(), N, NV, K, storage="bf16",
                        sif_k1=8, rescore_r=20, keep_exact=False)
    for a, b in zip(one.export_sif(), st.export_sif()):
        assert np.array_equal(a, b)
    st.close()
    one.close()


def test_streamed_build_order_and_state_errors(gpu_lib, data):
    import torch
    X, cb, Q, qoff = data
    lib = gpu_lib.load()
    prm = gpu_lib._Params(N, NV, D, K, gpu_lib._STORAGE["bf16"], 1, 5, 10, 0)
    h = ctypes.c_void_p()
    st = gpu_lib._stream()
    cbd = torch.from_numpy(cb).cuda()
    bad = gpu_lib._Params(N, NV, D, K, gpu_lib._STORAGE["bf16"], 1, 5, 10, 1)  # keep_exact
    assert lib.gift_build_begin(ctypes.byref(bad), gpu_lib._ptr(cbd), st, ctypes.byref(h)) == 1
    assert lib.gift_build_begin(ctypes.byref(prm), gpu_lib._ptr(cbd), st, ctypes.byref(h)) == 0
    try:
        xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        one = xd[:1]
        assert lib.gift_build_add(h, 2, gpu_lib._ptr(one), 0, 1, st) == 1          # pass 1 is open
        assert lib.gift_build_add(h, 1, gpu_lib._ptr(one), N, 1, st) == 1          # out of range
        assert lib.gift_build_add(h, 1, gpu_lib._ptr(one), 0, 1, st) == 0
        assert lib.gift_build_add(h, 1, gpu_lib._ptr(one), 0, 1, st) == 1          # shape 0 twice
        assert lib.gift_build_end_pass(h, 1, st) == 1                               # shapes missing
        ids = torch.zeros(1, 5, dtype=torch.int32, device="cuda")
        sc = torch.zeros(1, 5, dtype=torch.float32, device="cuda")
        qo = np.array([0, 64], np.int32)
        q = torch.from_numpy(Q[:64]).cuda()
        assert lib.gift_query(h, gpu_lib._ptr(q), gpu_lib._ptr(qo), 1, gpu_lib.MATCH_FIF, 5, gpu_lib._ptr(ids),
                              gpu_lib._ptr(sc), st) == 6                            # ESTATE
        for p in (1, 2, 3):
            f0 = 1 if p == 1 else 0
            assert lib.gift_build_add(h, p, gpu_lib._ptr(xd[f0:]), f0, N - f0, st) == 0
            assert lib.gift_build_end_pass(h, p, st) == 0
        assert lib.gift_build_add(h, 3, gpu_lib._ptr(one), 0, 1, st) == 6          # build complete
        assert lib.gift_query(h, gpu_lib._ptr(q), gpu_lib._ptr(qo), 1, gpu_lib.MATCH_FIF, 5, gpu_lib._ptr(ids),
                              gpu_lib._ptr(sc), st) == 0
    finally:
        lib.gift_destroy_index(h)
