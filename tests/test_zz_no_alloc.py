"""gift_rerank_noalloc: S-IF re-ranking without device allocation.

Callers whose free device memory is held by another allocator, or that must
not enter the CUDA allocator on a latency-critical path, cannot let the
library allocate scratch per call; this entry point runs the same re-ranking
kernels on a fixed buffer inside the library. Its results must equal those of
gift_rerank, call after call (the shared buffer keeps the previous call's
contents, so a second call checks that nothing stale leaks into the result),
and it must take no device memory: neither from the device's default memory
pool, where the library's per-call scratch comes from, nor at all.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from synth import shape_views, query_views, kmeans_codebook

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sif_case(gpu_lib):
    import torch
    N, Nv, D, C, K = 240, 16, 64, 12, 16
    X = shape_views(0, N, Nv, D, C, 1301, 4301)
    cb = kmeans_codebook(X.reshape(-1, D), K, 3301, 8)
    Q, qoff, _ = query_views(12, (16, 9), D, C, 2301, 4301, max_views=16)
    ix = gpu_lib.Index(torch.from_numpy(X).cuda(), torch.from_numpy(cb).cuda(), N, Nv, K, storage="f32",
                       sif_k1=10, keep_exact=False)
    ids, sc = ix.query(torch.from_numpy(Q).cuda(), qoff, mode="fif", topk=30)
    torch.cuda.synchronize()
    yield ix, ids, sc
    ix.close()


class _DefaultPool:
    """The current device's default memory pool, read through the driver API
    (CUmemPool_attribute values of cuda.h)."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8

    def __init__(self):
        import torch
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(z)) == 0


def _call(lib, ix, ids, sc, k1, topk, out_ids, out_sp):
    import torch
    B, n_cand = ids.shape
    return lib.gift_rerank_noalloc(ix._h, ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(sc.data_ptr()), B, n_cand,
                                   k1, topk, ctypes.c_void_p(out_ids.data_ptr()),
                                   ctypes.c_void_p(out_sp.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_rerank_equals_rerank_twice(gpu_lib, sif_case):
    import torch
    ix, ids, sc = sif_case
    lib = gpu_lib.load()
    ref_ids, ref_sp = ix.rerank(ids, sc, k1=10, topk=20)
    torch.cuda.synchronize()
    ref_ids, ref_sp = ref_ids.cpu().numpy(), ref_sp.cpu().numpy()
    for _ in range(2):
        out_ids = torch.full(ref_ids.shape, -7, dtype=torch.int32, device="cuda")
        out_sp = torch.full(ref_sp.shape, float("nan"), dtype=torch.float32, device="cuda")
        st = _call(lib, ix, ids, sc, 10, 20, out_ids, out_sp)
        assert st == 0, lib.gift_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(out_ids.cpu().numpy(), ref_ids)
        assert np.allclose(out_sp.cpu().numpy(), ref_sp, rtol=1e-5, atol=1e-6)


def test_noalloc_rejects_a_batch_beyond_its_buffer(gpu_lib, sif_case):
    import torch
    ix, ids, sc = sif_case
    lib = gpu_lib.load()
    B = 20000  # 20 * B * N bytes > 16 MiB at N = 240
    big_ids = ids[:1].repeat(B, 1).contiguous()
    big_sc = sc[:1].repeat(B, 1).contiguous()
    out_ids = torch.empty((B, 5), dtype=torch.int32, device="cuda")
    out_sp = torch.empty((B, 5), dtype=torch.float32, device="cuda")
    st = _call(lib, ix, big_ids, big_sc, 10, 5, out_ids, out_sp)
    assert st == 1 and b"scratch" in lib.gift_last_error()


def test_noalloc_rerank_takes_no_device_memory(gpu_lib, sif_case):
    """gift_rerank draws its scratch from the default pool (the pool's high watermark
    rises); two calls of gift_rerank_noalloc leave the watermark and the device's free
    memory as they were."""
    import torch
    ix, ids, sc = sif_case
    lib = gpu_lib.load()
    pool = _DefaultPool()
    out_ids = torch.empty((ids.shape[0], 20), dtype=torch.int32, device="cuda")
    out_sp = torch.empty((ids.shape[0], 20), dtype=torch.float32, device="cuda")
    assert _call(lib, ix, ids, sc, 10, 20, out_ids, out_sp) == 0  # first call on the device: set-up
    torch.cuda.synchronize()
    used = pool.get(pool.USED_MEM_CURRENT)
    pool.reset_high()
    ix.rerank(ids, sc, k1=10, topk=20, out=(out_ids, out_sp))
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) > used  # the control allocates per call
    torch.cuda.synchronize()
    pool.reset_high()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        assert _call(lib, ix, ids, sc, 10, 20, out_ids, out_sp) == 0, lib.gift_last_error()
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) <= used
    assert torch.cuda.mem_get_info()[0] == free0
