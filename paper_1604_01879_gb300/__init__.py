"""GB300 (sm_103a) implementation of GIFT's on-line query path.

A thin binding over the C ABI of ``libgift.so`` (declared in include/gift.h):
argument marshalling only. Every step of the path runs in the library's CUDA
kernels; PyTorch supplies device memory and the current stream. There is no
CPU fallback: without the built library every call raises.

    import paper_1604_01879_gb300 as gift
    ix = gift.Index(db, codebook, n_shapes=N, views_per_shape=64, n_codewords=K,
                    storage="bf16", rescore_r=200, sif_k1=50)
    ids, scores = ix.query(q, q_offsets, topk=100)            # Eq. 4 (F-IF)
    ids2, sprime = ix.rerank(ids, scores, k1=50, topk=100)     # S-IF (Eqs. 7-14)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "GiftError", "load", "lib_path", "Index", "match_forward", "match_backward", "GiftMatch",
    "F32", "BF16", "FP8_E4M3", "MATCH_EXACT", "MATCH_FIF", "Aca", "kmeans", "render_views",
]

F32, BF16, FP8_E4M3 = 0, 1, 2
MATCH_EXACT, MATCH_FIF = 0, 1
_STORAGE = {"f32": F32, "fp32": F32, "bf16": BF16, "fp8": FP8_E4M3, "fp8_e4m3": FP8_E4M3}
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED", 6: "ESTATE"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class GiftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "libgift.so")


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "n_shapes", "views_per_shape", "dim", "n_codewords", "storage", "query_ma", "sif_k1",
        "rescore_r", "keep_exact", "db_ma")]


class _Info(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("n_rows", ctypes.c_int64),
                ("n_lists_nonempty", ctypes.c_int32), ("max_list_len", ctypes.c_int32),
                ("n_runs", ctypes.c_int64), ("max_runs", ctypes.c_int32),
                ("max_sif_entry", ctypes.c_int32), ("n_entries", ctypes.c_int64),
                ("sif_shapes", ctypes.c_int32), ("sif_k1", ctypes.c_int32)]


class _Timing(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in (
        "assign_ms", "bucket_ms", "scan_ms", "combine_ms", "topk_ms", "rescore_ms", "rerank_ms",
        "total_ms")] + [("scan_bytes", ctypes.c_int64), ("rescore_bytes", ctypes.c_int64),
                        ("scan_pairs", ctypes.c_int64), ("assign_kernel_ms", ctypes.c_float),
                        ("scan_kernel_ms", ctypes.c_float), ("rescore_kernel_ms", ctypes.c_float),
                        ("assign_rows", ctypes.c_int64)] + [(n, ctypes.c_int64) for n in (
                            "rescore_items", "rescore_items_kept", "cand_pairs", "cand_rows", "rescore_rows_read")]


class _ServerParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "slots", "max_batch_queries", "max_batch_views", "topk", "rerank", "start_paused")] + [
        ("memory_budget", ctypes.c_int64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("completed", "failed", "batches", "queued")] + [
        (n, ctypes.c_float) for n in ("mean_batch", "p50_ms", "p99_ms", "max_ms", "queries_per_s")] + [
        (n, ctypes.c_int64) for n in ("admission_waits", "peak_in_flight_bytes", "budget_bytes", "max_batch_bytes",
                                      "slot_bytes")]


_P = ctypes.c_void_p
_I32, _I64 = ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "gift_build_index": (_I32, [ctypes.POINTER(_Params), _P, _P, _P, ctypes.POINTER(_P)]),
    "gift_destroy_index": (None, [_P]),
    "gift_set_rescore_depth": (_I32, [_P, _I32]),
    "gift_build_begin": (_I32, [ctypes.POINTER(_Params), _P, _P, ctypes.POINTER(_P)]),
    "gift_build_add": (_I32, [_P, _I32, _P, _I32, _I32, _P]),
    "gift_build_end_pass": (_I32, [_P, _I32, _P]),
    "gift_query": (_I32, [_P, _P, _P, _I32, _I32, _I32, _P, _P, _P]),
    "gift_rerank": (_I32, [_P, _P, _P, _I32, _I32, _I32, _I32, _P, _P, _P]),
    "gift_rerank_noalloc": (_I32, [_P, _P, _P, _I32, _I32, _I32, _I32, _P, _P, _P]),
    "gift_sif_from_neighbours": (_I32, [_P, _P, _P, _I32, _I32, _P]),
    "gift_merge_topk": (_I32, [_P, _P, _I32, _I64, _I32, _P, _P, _P]),
    "gift_assign": (_I32, [_P, _P, _I64, _I32, _P, _P]),
    "gift_render_views": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _I32, _P, _P]),
    "gift_kmeans": (_I32, [_P, _I64, _I32, _I32, _P, _I32, _P, _P]),
    "gift_aca_build": (_I32, [_P, _P, _I32, ctypes.c_float, _I32, _P, ctypes.POINTER(_P)]),
    "gift_aca_rerank": (_I32, [_P, _P, _P, _P, _P, _I32, _I32, _I32, _P, _P, _P]),
    "gift_aca_pairs": (_I32, [_P, ctypes.POINTER(_I64)]),
    "gift_aca_export": (_I32, [_P, _P, _P, _P, _P, _P]),
    "gift_aca_destroy": (None, [_P]),
    "gift_export_fif": (_I32, [_P, _P, _P, _P, _P]),
    "gift_export_sif": (_I32, [_P, _P, _P, _P, _P, _P]),
    "gift_index_info": (_I32, [_P, ctypes.POINTER(_Info)]),
    "gift_set_timing": (_I32, [_P, _I32]),
    "gift_get_timing": (_I32, [_P, ctypes.POINTER(_Timing)]),
    "gift_match_forward": (_I32, [_P, _P, _I32, _P, _I32, _I32, _P, _I32, _I32, _I32, _P, _P, _P]),
    "gift_match_backward": (_I32, [_P, _P, _I32, _P, _I32, _I32, _P, _I32, _I32, _I32, _P, _P, _P, _P, _P,
                                   _P]),
    "gift_server_create": (_I32, [_P, ctypes.POINTER(_ServerParams), ctypes.POINTER(_P)]),
    "gift_server_submit": (_I32, [_P, _P, _I32, ctypes.POINTER(_I64)]),
    "gift_server_wait": (_I32, [_P, _I64, _I32, _P, _P]),
    "gift_server_resume": (_I32, [_P]),
    "gift_server_stats": (_I32, [_P, ctypes.POINTER(_ServerStats)]),
    "gift_server_destroy": (None, [_P]),
    "gift_last_error": (ctypes.c_char_p, []),
    "gift_launch_count": (_I64, []),
    "gift_version": (_I32, []),
}
SYMBOLS = tuple(_SIGS)


def load(path: str | None = None):
    """Load libgift.so (built in-tree by ``build.build()``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgift.so not built ({path}); run paper_1604_01879_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise GiftError(status, _lib.gift_last_error().decode())


def _stream(stream=None):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Raw pointer of a torch tensor (device or host) or a numpy array (host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if not x.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _host_offsets(q_off):
    a = np.ascontiguousarray(np.asarray(
        q_off.cpu().numpy() if hasattr(q_off, "cpu") else q_off, dtype=np.int32))
    return a


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().gift_launch_count())


class Index:
    """A built GIFT index resident on the current CUDA device."""

    def __init__(self, db_feats, codebook, n_shapes: int, views_per_shape: int, n_codewords: int,
                 storage="f32", query_ma: int = 1, sif_k1: int = 0, rescore_r: int = 0,
                 keep_exact: bool = True, db_ma: int = 1, stream=None):
        lib = load()
        dim = int(codebook.shape[-1])
        self.params = _Params(int(n_shapes), int(views_per_shape), dim, int(n_codewords),
                              _STORAGE[storage] if isinstance(storage, str) else int(storage),
                              int(query_ma), int(sif_k1), int(rescore_r), int(bool(keep_exact)), int(db_ma))
        self._h = ctypes.c_void_p()
        _check(lib.gift_build_index(ctypes.byref(self.params), _ptr(db_feats), _ptr(codebook),
                                    _stream(stream), ctypes.byref(self._h)))
        self.n_shapes, self.views_per_shape, self.dim = int(n_shapes), int(views_per_shape), dim
        self.n_codewords, self.query_ma, self.sif_k1 = int(n_codewords), int(query_ma), int(sif_k1)
        self.rescore_r = int(rescore_r)

    @classmethod
    def streamed(cls, chunk_fn, codebook, n_shapes: int, views_per_shape: int, n_codewords: int,
                 chunk_shapes: int = 1024, storage="bf16", query_ma: int = 1, sif_k1: int = 0,
                 rescore_r: int = 0, db_ma: int = 1, stream=None):
        """Build an index from chunks in three passes (gift_build_begin / add / end_pass).

        chunk_fn(first_shape, n_shapes) returns the float32 views [n_shapes, N_v, D] of
        those shapes (host numpy or device tensor); it is called once per chunk per pass,
        so a seeded generator can regenerate chunks instead of holding the database.
        """
        lib = load()
        self = cls.__new__(cls)
        dim = int(codebook.shape[-1])
        self.params = _Params(int(n_shapes), int(views_per_shape), dim, int(n_codewords),
                              _STORAGE[storage] if isinstance(storage, str) else int(storage),
                              int(query_ma), int(sif_k1), int(rescore_r), 0, int(db_ma))
        self._h = ctypes.c_void_p()
        st = _stream(stream)
        _check(lib.gift_build_begin(ctypes.byref(self.params), _ptr(codebook), st, ctypes.byref(self._h)))
        self.n_shapes, self.views_per_shape, self.dim = int(n_shapes), int(views_per_shape), dim
        self.n_codewords, self.query_ma, self.sif_k1 = int(n_codewords), int(query_ma), int(sif_k1)
        self.rescore_r = int(rescore_r)
        try:
            for p in (1, 2, 3):
                if p == 3 and sif_k1 == 0:
                    break
                for first in range(0, n_shapes, chunk_shapes):
                    n = min(chunk_shapes, n_shapes - first)
                    x = chunk_fn(first, n)
                    if isinstance(x, np.ndarray):
                        x = np.ascontiguousarray(x, dtype=np.float32)
                    _check(lib.gift_build_add(self._h, p, _ptr(x), int(first), int(n), st))
                    del x
                import torch
                torch.cuda.empty_cache()  # the stores allocated at the end of pass 1 are large
                _check(lib.gift_build_end_pass(self._h, p, st))
        except BaseException:
            self.close()
            raise
        return self

    # -- queries -----------------------------------------------------------
    def query(self, q_feats, q_offsets, mode="fif", topk: int = 10, out=None, stream=None):
        """Top-k (ids int32, scores float32) [B, topk] of each query (Eq. 4 or Eq. 3)."""
        import torch
        offs = _host_offsets(q_offsets)
        B = len(offs) - 1
        m = MATCH_FIF if mode in ("fif", MATCH_FIF) else MATCH_EXACT
        if out is None:
            dev = q_feats.device if hasattr(q_feats, "device") and q_feats.is_cuda else torch.device("cuda")
            out = (torch.empty((B, topk), dtype=torch.int32, device=dev),
                   torch.empty((B, topk), dtype=torch.float32, device=dev))
        _check(load().gift_query(self._h, _ptr(q_feats), ctypes.c_void_p(offs.ctypes.data), B, m, int(topk),
                                 _ptr(out[0]), _ptr(out[1]), _stream(stream)))
        return out

    def rerank(self, cand_ids, cand_scores, k1: int | None = None, topk: int = 10, out=None, stream=None):
        """S-IF re-ranking of candidate rows: (ids int32, S' float32) [B, topk]."""
        import torch
        B, n_cand = cand_ids.shape
        k1 = self.sif_k1 if k1 is None else int(k1)
        if out is None:
            dev = cand_ids.device if hasattr(cand_ids, "is_cuda") and cand_ids.is_cuda else torch.device("cuda")
            out = (torch.empty((B, topk), dtype=torch.int32, device=dev),
                   torch.empty((B, topk), dtype=torch.float32, device=dev))
        _check(load().gift_rerank(self._h, _ptr(cand_ids), _ptr(cand_scores), int(B), int(n_cand), k1, int(topk),
                                  _ptr(out[0]), _ptr(out[1]), _stream(stream)))
        return out

    def assign(self, feats, ma: int = 1, stream=None):
        """Codewords [n, ma] (int32) of device rows ``feats`` (the quantiser)."""
        import torch
        n = feats.shape[0]
        out = torch.empty((n, ma), dtype=torch.int32, device=feats.device)
        _check(load().gift_assign(self._h, _ptr(feats), int(n), int(ma), _ptr(out), _stream(stream)))
        return out

    # -- inspection ----------------------------------------------------------
    def export_fif(self):
        """(db_codes [N*Nv*db_ma], list_offsets [K+1], list_rows [entries]) as numpy arrays."""
        n = int(self.info()["n_entries"])
        codes = np.empty(n, np.int32)
        off = np.empty(self.n_codewords + 1, np.int64)
        rows = np.empty(n, np.int32)
        _check(load().gift_export_fif(self._h, _ptr(codes), _ptr(off), _ptr(rows), _stream()))
        return codes, off, rows

    def export_sif(self):
        """(entry_offsets [N+1], entry_ids, entry_members uint32, card uint64 [N]) as numpy arrays;
        N and k1 are the S-IF's own (gift_index_info)."""
        info = self.info()
        N, k1 = info["sif_shapes"], info["sif_k1"]
        if N <= 0:
            raise GiftError(5, "index built without an S-IF")
        off = np.empty(N + 1, np.int64)
        ids = np.empty(N * k1, np.int32)
        mem = np.empty(N * k1, np.uint32)
        card = np.empty(N, np.uint64)
        _check(load().gift_export_sif(self._h, _ptr(off), _ptr(ids), _ptr(mem), _ptr(card), _stream()))
        return off, ids, mem, card

    def info(self) -> dict:
        i = _Info()
        _check(load().gift_index_info(self._h, ctypes.byref(i)))
        return {n: getattr(i, n) for n, _ in _Info._fields_}

    def set_sif(self, nbr_ids, nbr_scores, n_shapes_total: int, k1: int, stream=None):
        """Install the S-IF of a whole (sharded) database from its ranked neighbour rows
        [n_shapes_total, k1] (global ids and scores; gift_sif_from_neighbours)."""
        _check(load().gift_sif_from_neighbours(self._h, _ptr(nbr_ids), _ptr(nbr_scores), int(n_shapes_total),
                                               int(k1), _stream(stream)))
        self.sif_k1 = int(k1)

    def set_rescore_depth(self, r: int):
        """FP32 rescore depth of later queries (0 = scores of the list store alone)."""
        _check(load().gift_set_rescore_depth(self._h, int(r)))
        self.rescore_r = int(r)

    def set_timing(self, on: bool = True):
        _check(load().gift_set_timing(self._h, int(bool(on))))

    def timing(self) -> dict:
        t = _Timing()
        _check(load().gift_get_timing(self._h, ctypes.byref(t)))
        return {n: getattr(t, n) for n, _ in _Timing._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gift_destroy_index(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def merge_topk(ids, scores, k: int, out=None, stream=None):
    """The k best (id, score) pairs of each row by (score desc, id asc) (gift_merge_topk);
    ids int32 and scores float32 [B, n], id < 0 = empty. Returns (ids int32, scores float32) [B, k]."""
    import torch
    B, n = ids.shape
    if out is None:
        dev = ids.device if hasattr(ids, "is_cuda") and ids.is_cuda else torch.device("cuda")
        out = (torch.empty((B, k), dtype=torch.int32, device=dev), torch.empty((B, k), dtype=torch.float32, device=dev))
    _check(load().gift_merge_topk(_ptr(ids), _ptr(scores), int(B), int(n), int(k), _ptr(out[0]), _ptr(out[1]),
                                  _stream(stream)))
    return out


# ---------------------------------------------------------------- differentiation
def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError("matching inputs must be float32 or bfloat16 tensors")


def match_forward(q, q_offsets, p, W=None, stream=None):
    """S [B, Np] of Eq. 3 after the projection u = W q, and the saved argmax [sum V_q, Np] (int16)."""
    import torch
    offs = _host_offsets(q_offsets)
    Bq = len(offs) - 1
    Np, nv, din = p.shape
    dt = _dtype_code(q)
    if p.dtype != q.dtype or (W is not None and W.dtype != q.dtype):
        raise TypeError("q, p and W must share a dtype")
    dout = W.shape[0] if W is not None else din
    S = torch.empty((Bq, Np), dtype=torch.float32, device=q.device)
    am = torch.empty((q.shape[0], Np), dtype=torch.int16, device=q.device)
    _check(load().gift_match_forward(_ptr(q), ctypes.c_void_p(offs.ctypes.data), Bq, _ptr(p), Np, nv, _ptr(W),
                                     din, dout, dt, _ptr(S), _ptr(am), _stream(stream)))
    return S, am


def match_backward(q, q_offsets, p, W, grad_S, argmax, need=(True, True, True), stream=None):
    """(dW or None, dQ, dP) of sum(grad_S * S) through the saved argmax pair (FP32 gradients)."""
    import torch
    offs = _host_offsets(q_offsets)
    Bq = len(offs) - 1
    Np, nv, din = p.shape
    dt = _dtype_code(q)
    dout = W.shape[0] if W is not None else din
    f32 = dict(dtype=torch.float32, device=q.device)
    dW = torch.empty(W.shape, **f32) if (W is not None and need[0]) else None
    dQ = torch.empty(q.shape, **f32) if need[1] else None
    dP = torch.empty(p.shape, **f32) if need[2] else None
    _check(load().gift_match_backward(_ptr(q), ctypes.c_void_p(offs.ctypes.data), Bq, _ptr(p), Np, nv, _ptr(W), din,
                                      dout, dt, _ptr(grad_S.contiguous()), _ptr(argmax), _ptr(dW), _ptr(dQ), _ptr(dP),
                                      _stream(stream)))
    return dW, dQ, dP


def _autograd_function():
    import torch

    class GiftMatch(torch.autograd.Function):
        """S = GiftMatch.apply(q, q_offsets, p, W): Eq. 3 after u = W q, differentiable in q, p, W."""

        @staticmethod
        def forward(ctx, q, q_offsets, p, W):
            q = q.contiguous()
            p = p.contiguous()
            Wc = W.contiguous() if W is not None else None
            S, am = match_forward(q, q_offsets, p, Wc)
            ctx.save_for_backward(q, p, Wc if Wc is not None else torch.empty(0), am)
            ctx.q_offsets = _host_offsets(q_offsets)
            ctx.has_w = W is not None
            return S

        @staticmethod
        def backward(ctx, gS):
            q, p, W, am = ctx.saved_tensors
            W = W if ctx.has_w else None
            need = (ctx.has_w and ctx.needs_input_grad[3], ctx.needs_input_grad[0], ctx.needs_input_grad[2])
            dW, dQ, dP = match_backward(q, ctx.q_offsets, p, W, gS.float().contiguous(), am, need)
            cast = (lambda g, like: None if g is None else g.to(like.dtype))
            return cast(dQ, q), None, cast(dP, p), (cast(dW, W) if ctx.has_w else None)

    return GiftMatch


class _Lazy:
    def __getattr__(self, item):
        return getattr(_autograd_function(), item)


GiftMatch = _Lazy()


# ---------------------------------------------------------------- serving
def render_views(vertices, triangles, vert_off, tri_off, n_az: int = 8, n_el: int = 8, H: int = 224,
                 W: int = 224, out=None, stream=None):
    """Depth-buffer views of a batch of meshes (Sec. 2.1): float32 [M, n_az * n_el, H, W]."""
    import torch
    vo = np.ascontiguousarray(np.asarray(vert_off, np.int64))
    to = np.ascontiguousarray(np.asarray(tri_off, np.int64))
    M = len(vo) - 1
    if isinstance(vertices, np.ndarray):
        vertices = np.ascontiguousarray(vertices, dtype=np.float32)
    if isinstance(triangles, np.ndarray):
        triangles = np.ascontiguousarray(triangles, dtype=np.int32)
    if out is None:
        out = torch.empty((M, n_az * n_el, H, W), dtype=torch.float32, device="cuda")
    _check(load().gift_render_views(_ptr(vertices), _ptr(triangles), _ptr(vo), _ptr(to), M, int(n_az), int(n_el),
                                    int(H), int(W), _ptr(out), _stream(stream)))
    return out


def kmeans(X, init_rows, iters: int, out=None, stream=None):
    """Lloyd's k-means on the GPU (the off-line vocabulary): centres float32 [K, D].

    X: float32 [n, D] (device tensor or host array); init_rows: the K rows that start as centres.
    """
    import torch
    init = np.ascontiguousarray(np.asarray(init_rows, np.int32))
    n, D = int(X.shape[0]), int(X.shape[1])
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float32)
    K = len(init)
    if out is None:
        out = torch.empty((K, D), dtype=torch.float32, device="cuda")
    _check(load().gift_kmeans(_ptr(X), n, D, K, _ptr(init), int(iters), _ptr(out), _stream(stream)))
    return out


ACA_NONE, ACA_AUGMENT, ACA_CO_AUGMENT = 0, 1, 2
_ACA_MODES = {"none": ACA_NONE, "aug": ACA_AUGMENT, "co": ACA_CO_AUGMENT}


class Aca:
    """Re-ranking with two similarity measures (Eqs. 9-11) over two indices of the same shapes.

    mode: "none" (Eq. 7 per measure), "aug" (Eq. 10) or "co" (Eq. 11, the paper's default);
    the indices must stay open while this object is used.
    """

    def __init__(self, measure1: Index, measure2: Index, k2: int = 4, alpha: float = 0.5, mode="co",
                 stream=None):
        self.m1, self.m2 = measure1, measure2
        self.k1, self.k2, self.alpha = measure1.sif_k1, int(k2), float(alpha)
        self.mode = _ACA_MODES[mode] if isinstance(mode, str) else int(mode)
        self.n_shapes = measure1.n_shapes
        self._h = ctypes.c_void_p()
        _check(load().gift_aca_build(measure1._h, measure2._h, self.k2, self.alpha, self.mode, _stream(stream),
                                     ctypes.byref(self._h)))

    def rerank(self, cand1, cand2, topk: int = 10, out=None, stream=None):
        """cand1 / cand2: (ids, scores) [B, n_cand] from each measure's query; returns (ids, S') [B, topk]."""
        import torch
        ids1, sc1 = cand1
        ids2, sc2 = cand2
        B, n_cand = ids1.shape
        if out is None:
            dev = ids1.device if hasattr(ids1, "is_cuda") and ids1.is_cuda else torch.device("cuda")
            out = (torch.empty((B, topk), dtype=torch.int32, device=dev),
                   torch.empty((B, topk), dtype=torch.float32, device=dev))
        _check(load().gift_aca_rerank(self._h, _ptr(ids1), _ptr(sc1), _ptr(ids2), _ptr(sc2), int(B), int(n_cand),
                                      int(topk), _ptr(out[0]), _ptr(out[1]), _stream(stream)))
        return out

    def export(self):
        """(entry_offsets [N+1], entry_ids, entry_members uint32, card uint64 [N]) as numpy arrays."""
        n = ctypes.c_int64()
        _check(load().gift_aca_pairs(self._h, ctypes.byref(n)))
        off = np.empty(self.n_shapes + 1, np.int64)
        ids = np.empty(max(1, n.value), np.int32)
        mem = np.empty(max(1, n.value), np.uint32)
        card = np.empty(self.n_shapes, np.uint64)
        _check(load().gift_aca_export(self._h, _ptr(off), _ptr(ids), _ptr(mem), _ptr(card), _stream()))
        return off, ids[:n.value], mem[:n.value], card

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gift_aca_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop over a resident index (gift_server_*): continuous batching of
    queries with mixed view counts, memory-based admission, p50/p99 latency."""

    def __init__(self, index: Index, slots: int = 3, max_batch_queries: int = 256, max_batch_views: int = 256 * 64,
                 topk: int = 10, rerank: bool = True, start_paused: bool = False, memory_budget: int = 0):
        self.index = index
        self.topk = int(topk)
        self.dim = index.dim
        p = _ServerParams(int(slots), int(max_batch_queries), int(max_batch_views), int(topk), int(bool(rerank)),
                          int(bool(start_paused)), int(memory_budget))
        self._h = ctypes.c_void_p()
        _check(load().gift_server_create(index._h, ctypes.byref(p), ctypes.byref(self._h)))

    def submit(self, q_feats) -> int:
        """Queue one query (host float32 [n_views, D]); returns its ticket."""
        q = np.ascontiguousarray(q_feats, dtype=np.float32)
        t = ctypes.c_int64()
        _check(load().gift_server_submit(self._h, ctypes.c_void_p(q.ctypes.data), int(q.shape[0]), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        """(ids int32 [topk], scores float32 [topk]) of a request; GiftError ETIMEOUT if not done in time."""
        ids = np.empty(self.topk, np.int32)
        sc = np.empty(self.topk, np.float32)
        _check(load().gift_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.c_void_p(ids.ctypes.data),
                                       ctypes.c_void_p(sc.ctypes.data)))
        return ids, sc

    def resume(self):
        _check(load().gift_server_resume(self._h))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load().gift_server_stats(self._h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gift_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
