"""Seeded view-feature workloads shaped like the paper's retrieval benchmarks.

Recipe (the paper uses CNN activations of 64 depth views per shape, L2-normalised,
Sec. 2.2 and Sec. 3; those features and datasets are not available, so these
stand in for them):

* class centres mu_c ~ N(0, I_D), c = 0..C-1, drawn from the centre seed;
* shape s belongs to class s mod C; each of its views is
  v = ReLU(mu_c + noise * eps), eps ~ N(0, I_D) -- non-negative like ReLU
  activations -- then L2-normalised in float64 and rounded to float32;
* queries are drawn with the same centres from a different seed stream;
* every block of ``BLOCK`` shapes has its own generator keyed by (seed, block),
  so any shape range can be regenerated alone and in any order, in parallel.

The codebook fixture (the vocabulary B of Sec. 2.3) is trained off-line by a
seeded Lloyd k-means on a seeded sample of database views. The method treats
the codebook as an input; this module only prepares it.

Nothing here computes a matching score, a quantisation used by the method, a
ranking or a re-ranking.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

BLOCK = 16  # shapes per independently seeded generator block


@dataclass(frozen=True)
class Config:
    """One synthetic workload (sizes of the paper-shaped benchmark it stands in for)."""

    name: str
    n_shapes: int          # N, database shapes
    n_views: int           # N_v, database views per shape
    dim: int               # D, feature dimension
    n_classes: int
    n_codewords: int       # K, F-IF vocabulary size
    n_queries: int
    query_views: tuple = (64,)   # view counts a query draws from (uniformly)
    query_ma: int = 1      # query-side multiple assignment
    storage: str = "f32"   # F-IF feature store: f32 | bf16 | fp8
    rescore_r: int = 0     # FP32 rescore depth (0 = off)
    topk: int = 10
    sif_k1: int = 10
    batch: int = 0         # queries per gift_query call (0 = all)
    kmeans_shapes: int = 0 # shapes sampled for the codebook (0 = all)
    kmeans_iters: int = 25
    noise: float = 0.3
    seed: int = 0          # config number; seeds derive from it
    generator: str = "sequential"  # "sequential" (numpy PCG64 blocks) | "counter" (synth.counter)
    extra: dict = field(default_factory=dict)

    @property
    def db_seed(self) -> int:
        return 1000 + self.seed

    @property
    def query_seed(self) -> int:
        return 2000 + self.seed

    @property
    def codebook_seed(self) -> int:
        return 3000 + self.seed

    @property
    def centre_seed(self) -> int:
        return 4000 + self.seed


CONFIGS = {
    # WM-SHREC07-sized database (400 models / 20 classes in the paper, Sec. 3.3)
    "db200x64_d128_k64": Config(
        name="db200x64_d128_k64", n_shapes=200, n_views=64, dim=128, n_classes=20,
        n_codewords=64, n_queries=10, storage="f32", rescore_r=0, topk=10,
        sif_k1=10, seed=1),
    # ModelNet40-sized database (12,311 models / 40 classes, Sec. 3.1)
    "db12000x64_d4096_k1024": Config(
        name="db12000x64_d4096_k1024", n_shapes=12000, n_views=64, dim=4096,
        n_classes=40, n_codewords=1024, n_queries=1000, storage="bf16",
        rescore_r=200, topk=100, sif_k1=50, kmeans_shapes=256, kmeans_iters=10,
        seed=2),
    # reduced ModelNet40-shaped case for kernel profiles (lists > L2, few GB on device)
    "db2000x64_d4096_k1024": Config(
        name="db2000x64_d4096_k1024", n_shapes=2000, n_views=64, dim=4096,
        n_classes=40, n_codewords=1024, n_queries=256, storage="bf16",
        rescore_r=200, topk=100, sif_k1=50, kmeans_shapes=256, kmeans_iters=10,
        seed=5),
    # reduced case of the FP8 / MA = 2 configuration for kernel profiles (~4 GB on the device,
    # list stores larger than L2) with the large one's list structure: 8 codewords per class,
    # ~8 query slots per list (32-query batches), candidates of about two classes per query
    "db3200x64_d4096_k512_fp8": Config(
        name="db3200x64_d4096_k512_fp8", n_shapes=3200, n_views=64, dim=4096, n_classes=64, n_codewords=512,
        n_queries=256, query_ma=2, storage="fp8", rescore_r=100, topk=100, sif_k1=50, batch=32,
        kmeans_shapes=128, kmeans_iters=6, seed=6, generator="counter"),
    # the 200,000-shape workload with a tenth of the shapes per class (same classes, vocabulary, batch, MA), rescore
    # depth scaled with the database: the same list and slot structure per batch at 26 GB, for DRAM counters
    "db20000x64_d4096_k4096_fp8": Config(
        name="db20000x64_d4096_k4096_fp8", n_shapes=20000, n_views=64,
        dim=4096, n_classes=400, n_codewords=4096, n_queries=256, query_ma=2,
        storage="fp8", rescore_r=100, topk=100, sif_k1=50, batch=256,
        kmeans_shapes=512, kmeans_iters=6, seed=3, generator="counter"),
    # 16x scale-up of ModelNet40 with FP8 store and query-side MA = 2
    "db200000x64_d4096_k4096_fp8": Config(
        name="db200000x64_d4096_k4096_fp8", n_shapes=200000, n_views=64,
        dim=4096, n_classes=400, n_codewords=4096, n_queries=10000, query_ma=2,
        storage="fp8", rescore_r=1000, topk=100, sif_k1=50, batch=256,
        kmeans_shapes=512, kmeans_iters=6, seed=3, generator="counter"),
}


def second_measure(cfg: Config) -> Config:
    """A second feature set of the same shapes, standing in for the paper's second CNN layer
    (Sec. 3 uses two layers): same shapes, views and classes, half the dimension, its own
    centres, noise, queries and codebook (seeds shifted by 50)."""
    import dataclasses
    return dataclasses.replace(cfg, name=cfg.name + "_m2", dim=max(16, cfg.dim // 2), seed=cfg.seed + 50,
                               query_views=(cfg.n_views,))


def _gen(seed: int, block: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(block)])


def class_centres(n_classes: int, dim: int, seed: int) -> np.ndarray:
    """mu_c ~ N(0, I_D), float64 [C, D]."""
    return _gen(seed, 0).standard_normal((n_classes, dim))


def _fill_views(out, first_shape, n_shapes, n_views, centres, seed, noise, labels):
    """Views of shapes [first_shape, first_shape + n_shapes) into out[...]."""
    C, D = centres.shape
    b0 = first_shape // BLOCK
    b1 = (first_shape + n_shapes + BLOCK - 1) // BLOCK
    for b in range(b0, b1):
        g = _gen(seed, b + 1)
        s_lo, s_hi = b * BLOCK, (b + 1) * BLOCK
        eps = g.standard_normal((BLOCK, n_views, D))
        lo = max(s_lo, first_shape)
        hi = min(s_hi, first_shape + n_shapes)
        for s in range(lo, hi):
            cls = labels(s) % C
            v = centres[cls][None, :] + noise * eps[s - s_lo]
            np.maximum(v, 0.0, out=v)
            nrm = np.sqrt((v * v).sum(axis=1, keepdims=True))
            nrm[nrm == 0] = 1.0
            out[s - first_shape] = (v / nrm).astype(np.float32)


def shape_views(first_shape: int, n_shapes: int, n_views: int, dim: int,
                n_classes: int, seed: int, centre_seed: int, noise: float = 0.3,
                threads: int | None = None) -> np.ndarray:
    """Database views of shapes [first_shape, first_shape+n_shapes): float32 [n, Nv, D].

    Shape s has class s mod n_classes.
    """
    centres = class_centres(n_classes, dim, centre_seed)
    out = np.empty((n_shapes, n_views, dim), np.float32)
    threads = threads or min(32, os.cpu_count() or 1)
    # spans of whole generator blocks, so each block is drawn by one worker
    end = first_shape + n_shapes
    b0, b1 = first_shape // BLOCK, (end + BLOCK - 1) // BLOCK
    spans = []
    for b in range(b0, b1, 4):
        lo = max(b * BLOCK, first_shape)
        hi = min((b + 4) * BLOCK, end)
        if hi > lo:
            spans.append((lo, hi))

    def work(span):
        lo, hi = span
        _fill_views(out[lo - first_shape:hi - first_shape], lo, hi - lo, n_views,
                    centres, seed, noise, lambda s: s)

    if threads == 1 or len(spans) == 1:
        for sp in spans:
            work(sp)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, spans))
    return out


def signed_views(n_shapes: int, n_views: int, dim: int, n_classes: int, seed: int, centre_seed: int,
                 weight: float = 0.5) -> np.ndarray:
    """Signed view features for edge cases the ReLU recipe never reaches: float32 [n, N_v, D].

    v = weight * mu_c + eps with mu_c, eps ~ N(0, I_D) and no ReLU, L2-normalised in
    float64 and rounded to float32; shape s has class s mod n_classes. Cosines of
    such views take both signs.
    """
    centres = class_centres(n_classes, dim, centre_seed)
    eps = _gen(seed, 1).standard_normal((n_shapes, n_views, dim))
    v = weight * centres[np.arange(n_shapes) % n_classes][:, None, :] + eps
    v /= np.sqrt((v * v).sum(axis=2, keepdims=True))
    return v.astype(np.float32)


def config_views(cfg: Config, first: int, n: int, device=None, query: bool = False):
    """Views of shapes [first, first + n) of a config's database (or query set).

    float32 [n, N_v, D]: a numpy array, or a torch tensor drawn on ``device``
    (counter generator only; bit-identical to the host draw).
    """
    seed = cfg.query_seed if query else cfg.db_seed
    if cfg.generator == "counter":
        from .counter import shape_views_np, shape_views_torch
        if device is not None:
            return shape_views_torch(first, n, cfg.n_views, cfg.dim, cfg.n_classes, seed, cfg.centre_seed,
                                     device=device)
        return shape_views_np(first, n, cfg.n_views, cfg.dim, cfg.n_classes, seed, cfg.centre_seed)
    if device is not None:
        raise ValueError("only the counter generator draws on a device")
    return shape_views(first, n, cfg.n_views, cfg.dim, cfg.n_classes, seed, cfg.centre_seed, cfg.noise)


def query_views(n_queries: int, view_choices, dim: int, n_classes: int,
                seed: int, centre_seed: int, noise: float = 0.3,
                max_views: int = 64, generator: str = "sequential"):
    """Query views: (float32 [sum V_q, D], int32 offsets [B+1], int64 classes [B]).

    Query b has class b mod n_classes; its view count is drawn uniformly from
    ``view_choices`` (a seeded draw); its views are the first V_q views of a
    ``max_views``-view draw from the recipe.
    """
    view_choices = tuple(int(v) for v in view_choices)
    counts = _gen(seed, 0).choice(np.asarray(view_choices), size=n_queries) \
        if len(view_choices) > 1 else np.full(n_queries, view_choices[0])
    nv = max(max_views, max(view_choices))
    if generator == "counter":
        from .counter import shape_views_np
        full = shape_views_np(0, n_queries, nv, dim, n_classes, seed, centre_seed)
    else:
        full = shape_views(0, n_queries, nv, dim, n_classes, seed, centre_seed, noise)
    offs = np.zeros(n_queries + 1, np.int64)
    offs[1:] = np.cumsum(counts)
    flat = np.empty((int(offs[-1]), dim), np.float32)
    for b in range(n_queries):
        flat[offs[b]:offs[b + 1]] = full[b, :counts[b]]
    classes = np.arange(n_queries) % n_classes
    return flat, offs.astype(np.int32), classes


def kmeans_init_rows(n: int, k: int, seed: int) -> np.ndarray:
    """The fixture's initial centres: a seeded choice of k distinct rows of n, ascending (int32 [k])."""
    return np.sort(_gen(seed, 0).choice(n, size=k, replace=False)).astype(np.int32)


def kmeans_codebook(sample: np.ndarray, k: int, seed: int, iters: int) -> np.ndarray:
    """Seeded Lloyd k-means fixture on ``sample`` (float [n, D]) -> float32 [k, D].

    Initial centres are a seeded choice of k distinct sample points; a cluster
    that empties is re-seeded with the point farthest from its centre. The
    paper trains its vocabulary off-line with k-means but gives no details.
    """
    X = np.asarray(sample, np.float64)
    n = X.shape[0]
    if k > n:
        raise ValueError("k-means needs at least k sample points")
    C = X[kmeans_init_rows(n, k, seed)].copy()
    X32 = X.astype(np.float32)
    xx = (X * X).sum(1)
    for _ in range(iters):
        cc = (C * C).sum(1)
        dist = xx[:, None] - 2.0 * (X32 @ C.T.astype(np.float32)) + cc[None, :]
        lab = dist.argmin(1)
        order = np.argsort(lab, kind="stable")
        cnt = np.bincount(lab, minlength=k)
        starts = np.concatenate([[0], np.cumsum(cnt)[:-1]])
        nonempty = cnt > 0
        sums = np.zeros_like(C)
        sums[nonempty] = np.add.reduceat(X[order], starts[nonempty], axis=0)
        far = np.argsort(-dist[np.arange(n), lab], kind="stable")
        fi = 0
        for c in range(k):
            if cnt[c] > 0:
                C[c] = sums[c] / cnt[c]
            else:
                C[c] = X[far[fi]]
                fi += 1
    return C.astype(np.float32)


def projection_matrix(d_out: int, d_in: int, seed: int, std: float) -> np.ndarray:
    """Seeded Gaussian initialisation of a linear view projection, float32 [d_out, d_in]."""
    return (_gen(seed, 0).standard_normal((d_out, d_in)) * std).astype(np.float32)


def upstream_grad(rows: int, cols: int, seed: int) -> np.ndarray:
    """Seeded N(0, 1) upstream gradient dL/dS, float32 [rows, cols]."""
    return _gen(seed, 0).standard_normal((rows, cols)).astype(np.float32)


# differentiation workload: 256 query shapes x 64 views against 4,096 database
# shapes x 64 views, D = 4096, BF16, projection 4096 -> 512 with std 1/64
DIFF_WORKLOAD = dict(name="match256x4096x64_d4096_p512_bf16", n_queries=256, n_shapes=4096, n_views=64,
                     dim=4096, d_out=512, w_std=1.0 / 64, n_classes=40, seed=4)


def make_config_inputs(cfg: Config, with_db: bool = True, n_queries: int | None = None):
    """Database views, codebook and queries of a config as float32 arrays.

    Returns dict(db [N, Nv, D] or None, codebook [K, D], q [sum V_q, D],
    q_off [B+1], q_class [B]).
    """
    nq = cfg.n_queries if n_queries is None else n_queries
    db = None
    if with_db and cfg.generator == "counter":
        db = config_views(cfg, 0, cfg.n_shapes)
    elif with_db:
        db = shape_views(0, cfg.n_shapes, cfg.n_views, cfg.dim, cfg.n_classes,
                         cfg.db_seed, cfg.centre_seed, cfg.noise)
    codebook = config_codebook(cfg, db)
    q, q_off, q_cls = query_views(nq, cfg.query_views, cfg.dim, cfg.n_classes,
                                  cfg.query_seed, cfg.centre_seed, cfg.noise,
                                  max_views=cfg.n_views, generator=cfg.generator)
    return dict(db=db, codebook=codebook, q=q, q_off=q_off, q_class=q_cls)


def codebook_sample_shapes(cfg: Config) -> np.ndarray:
    """The database shapes whose views train the codebook fixture (seeded, ascending)."""
    ks = cfg.kmeans_shapes or cfg.n_shapes
    if ks >= cfg.n_shapes:
        return np.arange(cfg.n_shapes)
    return np.sort(_gen(cfg.codebook_seed, 1).choice(cfg.n_shapes, ks, replace=False))


def config_codebook(cfg: Config, db=None) -> np.ndarray:
    """The codebook fixture of a config: seeded k-means on a seeded sample of its database shapes."""
    sample_shapes = codebook_sample_shapes(cfg)
    if db is not None:
        sample = db[sample_shapes].reshape(-1, cfg.dim)
    elif cfg.generator == "counter":
        from .counter import centres_np, key_of, _views_np
        mu, key = centres_np(cfg.n_classes, cfg.dim, cfg.centre_seed), key_of(cfg.db_seed)
        with ThreadPoolExecutor(min(32, os.cpu_count() or 1)) as ex:
            parts = list(ex.map(lambda s: _views_np(int(s), 1, cfg.n_views, cfg.dim, mu, key), sample_shapes))
        sample = np.concatenate(parts).reshape(-1, cfg.dim)
    else:
        sample = np.concatenate([
            shape_views(int(s), 1, cfg.n_views, cfg.dim, cfg.n_classes, cfg.db_seed,
                        cfg.centre_seed, cfg.noise, threads=1) for s in sample_shapes
        ]).reshape(-1, cfg.dim)
    return kmeans_codebook(sample, cfg.n_codewords, cfg.codebook_seed, cfg.kmeans_iters)
