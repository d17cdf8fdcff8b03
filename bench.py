"""Benchmark of the GIFT query path on GB300.

One step = one batch of queries through the whole hot path: quantise the
query views, bucket them by codeword, scan the touched F-IF lists, combine
into shape scores (Eq. 4), select the top-R, rescore them with FP32
features, select the top-k (gift_query), then re-rank through the S-IF
(gift_rerank, Eqs. 7-14).

Default workload: 12,000 database shapes x 64 views x D=4096 (BF16 store),
K=1024 codewords, batches of 1,000 queries of 64 views, FP32 rescore of the
top 200, top-100 output, S-IF k1=50.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gift|reference]

Under torchrun (N > 1) every rank holds a replica of the index and serves
its own query batches (queries are independent; no data-path collective):
weak scaling, time = max over ranks.

``--config db200000x64_d4096_k4096_fp8`` measures the 200,000-shape FP8
index instead (streamed build from a device-side generator, batches of 256
queries, MA = 2); its recall@100 comes from the oracle's bounded top-k of
Eq. 4, computed in a separate process on the host cores meanwhile.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_CONFIG = "db200000x64_d4096_k4096_fp8"
SECOND_CONFIG = "db12000x64_d4096_k1024"
METRIC = "queries/s and p99 ms, F-IF vs exact on one GB300, at recall@100 >= 0.99 vs FP64"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.t0 = time.time()
        self.marks = []

    def mark(self):
        self.marks.append(time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip() for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            c = [x.strip() for x in r.split(",")]
            try:
                s, m = float(c[1]), float(c[2])
            except (ValueError, IndexError):
                continue
            mx = max(mx, m)
            sm.append(s)
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        busy = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- peaks / traffic
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1604_01879_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, src_hash: str):
    """DRAM bytes per unit of work from the committed ncu summary (captured on a reduced
    case of the same kernel), while the kernel's source is unchanged since the capture:
    (bytes per unit, unit, capture workload), or (None, None, None)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        for line in open(path):
            c = [x.strip() for x in line.strip().strip("|").split("|")]
            if len(c) >= 5 and c[0] == kernel and c[1] == src_hash:
                return float(c[3]), c[4], c[2]
    except (OSError, ValueError):
        pass
    return None, None, None


# ---------------------------------------------------------------- reference arm
def cpu_oracle_run(cfg, data, n_queries, steps, db_codes=None):
    """Time the FP64 oracle's query path (Eq. 4 + ranking + S-IF re-rank) on host cores."""
    from oracle import gift_oracle as O
    N, Nv, D = cfg.n_shapes, cfg.n_views, cfg.dim
    X = data["db"]
    if db_codes is None:
        t = time.time()
        db_codes = O.quantize(X.reshape(-1, D), data["codebook"], 1).reshape(N, Nv)
        log(f"[reference] oracle database codes in {time.time() - t:.1f}s")
    # S-IF activations of the database: a seeded sparse stand-in with k1 entries per row
    # (building the true ones needs N oracle queries, an off-line cost outside the step)
    g = np.random.default_rng(cfg.seed + 77)
    F_db = np.zeros((N, N))
    for p in range(N):
        nb = g.choice(N, cfg.sif_k1, replace=False)
        F_db[p, nb] = g.random(cfg.sif_k1)
        F_db[p, p] = 1.0
    q, qoff = data["q"], data["q_off"]
    times = []
    b = 0
    for _ in range(steps):
        t = time.time()
        for _ in range(n_queries):
            lo, hi = qoff[b], qoff[b + 1]
            Qb = q[lo:hi]
            off = np.array([0, hi - lo])
            qc = O.quantize(Qb, data["codebook"], cfg.query_ma)
            S = O.fif_scores(Qb, off, qc, X, db_codes)[0]
            O.rank(S, cfg.topk)
            O.rerank(S[None, :], F_db, cfg.sif_k1, cfg.topk)
            b = (b + 1) % (len(qoff) - 1)
        times.append(time.time() - t)
    return times, db_codes


def oracle_bounded_worker(cfg_name, q_ids, codebook, k, threads, conn):
    """Spawned process: the oracle's top-k of Eq. 4 for sampled queries of a
    counter-generated config (bound pass over every database shape, then the
    pruned walk), timed on the host cores."""
    from synth import CONFIGS
    from synth.counter import shape_views_np
    from oracle import gift_oracle as O
    cfg = CONFIGS[cfg_name]
    try:
        t0 = time.time()
        Q = np.concatenate([shape_views_np(int(b), 1, cfg.n_views, cfg.dim, cfg.n_classes, cfg.query_seed,
                                           cfg.centre_seed, threads=1)[0] for b in q_ids])
        off = np.arange(len(q_ids) + 1) * cfg.n_views
        qc = O.quantize(Q, codebook, cfg.query_ma)

        def views_of(f, n):
            return shape_views_np(f, n, cfg.n_views, cfg.dim, cfg.n_classes, cfg.db_seed, cfg.centre_seed,
                                  threads=threads)

        U = O.fif_upper_bound(Q, off, views_of, cfg.n_shapes, chunk_shapes=512)
        t1 = time.time()
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            def group(ids):
                return np.stack(list(ex.map(lambda p: views_of(int(p), 1)[0], ids)))
            res, visited = O.fif_topk_bounded(Q, off, qc, codebook, lambda p: views_of(p, 1)[0], U, k,
                                              views_of_group=group)
        conn.send({"ids": [r[0].tolist() for r in res], "scores": [r[1].tolist() for r in res],
                   "visited": visited, "bound_s": t1 - t0, "walk_s": time.time() - t1,
                   "seconds": time.time() - t0, "threads": threads})
    except Exception as e:  # reported by the parent
        conn.send({"error": repr(e)})
    conn.close()


def roofline(cfg, st, scan_pairs, scan_bytes, rescore_bytes, assign_rows, peaks, peak_src, with_traffic=True,
             cand=None):
    """Roofline entry of the dominant kernel (most device time per step), from the
    per-kernel CUDA-event times ``st`` and the batch's work counters. ``cand`` (the
    library's candidate counters: cand_pairs, cand_rows, rescore_items, rescore_items_kept,
    rescore_rows_read) makes the separate rescore's work its candidates' pairs and rows."""
    bf16_peak = float(peaks["bf16_tflops"])
    hbm_peak = float(peaks["hbm_gbs"])
    D = cfg.dim
    # useful tensor-core FLOPs (unpadded pairs):
    #   scan     2 * pairs * D                       (one product)
    #   rescore  3 * 2 * pairs * D                   (hi*hi + hi*lo + lo*hi, FP32-accurate)
    #   assign   3 * 2 * rows * K * D                (same split)
    # the FP8 scan runs kind::f8f6f4 MMAs: its peak is the BF16 peak x 2 (nominal ratio)
    scan_peak = bf16_peak * (2.0 if cfg.storage == "fp8" else 1.0)
    # algorithmic bytes:
    #   scan     every touched list row once per batch (store row + id + scale)
    #   rescore  every touched list row once per batch (two-part BF16 row + id + scale)
    #   assign   the FP32 query rows and the FP32 codebook once
    # a BF16 store with its two-part rows runs scan and rescore as one fused pass
    # (three products over every touched pair, reported as the rescore kernel)
    fused = cfg.storage == "bf16" and st["scan_kernel_ms"] <= 0 and st["rescore_kernel_ms"] > 0
    resc_name = "fused scan + rescore" if fused else "rescore"
    # the launches behind each timed role (lists of up to 80 query slots run with the
    # entries as MMA rows, one launch per slot tile of 16, 32, 64 or 80)
    classes = ["16", "32", "64", "80"]
    launches = {
        "scan": (["tc_engine<ScanPolicy<1>>"] + [f"tc_engine<SlotsPolicy<1,1,{c}>>" for c in classes]
                 if cfg.storage == "fp8" else ["tc_engine<ScanPolicy<2>>"]),
        "rescore": ["tc_engine<RescorePolicy>"] + [f"tc_engine<SlotsPolicy<2,3,{c}>>" for c in classes],
        "fused scan + rescore": ["tc_engine<RescorePolicy> (every touched pair, FP32 level)"],
        "quantiser": ["tc_engine<AssignPolicy>"],
    }
    resc_flops, resc_bytes = 6.0 * scan_pairs * D, rescore_bytes
    if cand and not fused:
        # the rescore runs the work items holding candidate runs; its work is the
        # candidates' (slot, entry) pairs and the candidate rows, each read once
        resc_flops, resc_bytes = 6.0 * cand["cand_pairs"] * D, cand["cand_rows"] * (4.0 * D + 12)
    kernels = {
        "scan": (st["scan_kernel_ms"], 2.0 * scan_pairs * D, scan_bytes, ["k_scan_tc.cu"], scan_peak),
        resc_name: (st["rescore_kernel_ms"], resc_flops, resc_bytes, ["k_scan_tc.cu"], bf16_peak),
        "quantiser": (st["assign_kernel_ms"], 6.0 * assign_rows * cfg.n_codewords * D,
                      assign_rows * D * 4 + cfg.n_codewords * D * 4, ["k_assign.cu"], bf16_peak),
    }
    # each kernel against both roofs; its bound is the roof it is closer to
    table = {}
    for name, (ms, flops, nbytes, files, pk) in kernels.items():
        if ms > 0:
            ach = flops / (ms / 1e3) / 1e12
            gbs = nbytes / (ms / 1e3) / 1e9
            t_frac, h_frac = ach / pk, gbs / hbm_peak
            if h_frac > t_frac:
                table[name] = {"ms": ms, "bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                               "frac": h_frac, "tensor_frac": t_frac}
            else:
                table[name] = {"ms": ms, "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                               "frac": t_frac, "hbm_frac": h_frac}
            table[name]["launches"] = launches[name]
    if not table:  # no engine kernel ran (FP32 store scanned on the CUDA cores, no tensor-core quantiser)
        return None
    dom = max(table, key=lambda k: table[k]["ms"])
    src_hash = kernel_source_hash(kernels[dom][3] + ["tc_engine.cuh", "tc_common.cuh"])
    per_unit, unit, capture = recorded_traffic(dom, src_hash) if with_traffic else (None, None, None)
    # units of this launch: rows of the touched lists (scan, fused pass), rows the rescore reads,
    # rows quantised
    eb = 1 if cfg.storage == "fp8" else (2 if cfg.storage == "bf16" else 4)
    units = {"touched row": scan_bytes / (D * eb + 12.0),
             "rescore row read": (cand or {}).get("rescore_rows_read"),
             "row quantised": assign_rows}.get(unit)
    traffic = per_unit * units if per_unit is not None and units else None
    dt = table[dom]
    if dt["bound"] == "hbm":
        psrc = f"{peak_src} hbm_gbs"
        work = "algorithmic bytes: every list row the batch touches, read once"
    else:
        psrc = f"{peak_src} bf16_tflops (burst)" + (" x 2 for E4M3" if dt["peak"] != bf16_peak else "")
        work = ("useful MMA FLOPs on unpadded pairs; the rescore (or fused scan + rescore) and quantiser run "
                "three BF16 products per FP32-accurate product")
    if dom == "rescore" and cand:
        work = "algorithmic bytes: the candidate rows (two-part BF16 row + id + scale) of the touched lists, read once"
    out = {"kernel": dom, "launches": dt["launches"], "bound": dt["bound"], "achieved": dt["achieved"], "peak": dt["peak"],
           "unit": dt["unit"], "frac": dt["frac"], "traffic": traffic,
           "traffic_source": (f"ncu dram__bytes_read + write on {capture}: {per_unit:.4g} B per {unit}, x {units:.4g}"
                              if traffic is not None else None),
           "peak_source": psrc,
           "kernel_ms": dt["ms"], "work": work, "src_hash": src_hash, "all": table,
           "scan_hbm": {"algorithmic_bytes": scan_bytes,
                        "achieved_gbs": (scan_bytes / (st["scan_kernel_ms"] / 1e3) / 1e9
                                         if st["scan_kernel_ms"] > 0 else None),
                        "peak_gbs": hbm_peak}}
    if cand and cand.get("rescore_items"):
        c = dict(cand)
        c["items_kept_fraction"] = cand["rescore_items_kept"] / cand["rescore_items"]
        c["candidate_pair_fraction"] = cand["cand_pairs"] / max(scan_pairs, 1)
        if fused and st["rescore_kernel_ms"] > 0:
            # the method needs one BF16 product per touched pair (the Eq. 4 scan) and
            # three only on candidate pairs (the FP32 rescore)
            mflops = 2.0 * scan_pairs * D + 6.0 * cand["cand_pairs"] * D
            c["method_work_frac"] = mflops / (st["rescore_kernel_ms"] / 1e3) / 1e12 / bf16_peak
        out["candidate_work"] = c
    return out


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] or [os.cpu_count() or 1])
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# ---------------------------------------------------------------- oracle on a slice (large configs)
def cpu_oracle_slice(cfg, steps, codebook, n_slice=1000):
    """The FP64 oracle, as it stands, on a bounded sample of a counter-generated
    config: each step is one query against a contiguous slice of ``n_slice``
    database shapes -- its views quantised (``quantize``), Eq. 4 literally over
    the slice (``fif_scores``; the slice's database codes are computed first and
    untimed, like the off-line codes of the smaller configs), its top-k
    (``rank``) and the S-IF re-rank through the oracle's inverted file (Eqs. 13
    and 14, ``sif_scores_inverted``) over a seeded stand-in activation of the
    slice. Returns the per-step seconds; one step covers n_slice / N of a query."""
    from synth import config_views
    from oracle import gift_oracle as O
    Nv, D = cfg.n_views, cfg.dim
    t0 = time.time()
    X = config_views(cfg, 0, n_slice)
    dbc = O.quantize(X.reshape(-1, D), codebook, 1).reshape(n_slice, Nv)
    g = np.random.default_rng(cfg.seed + 77)
    F_db = np.zeros((n_slice, n_slice))
    for p in range(n_slice):
        F_db[p, g.choice(n_slice, cfg.sif_k1, replace=False)] = g.random(cfg.sif_k1)
        F_db[p, p] = 1.0
    card, entries = O.build_sif(F_db)
    Qall = config_views(cfg, 0, steps, query=True)
    log(f"[oracle slice] {n_slice} shapes prepared in {time.time() - t0:.1f}s")
    off = np.array([0, Nv])
    times = []
    for s_ in range(steps):
        Qb = Qall[s_]
        t = time.time()
        S = O.fif_scores(Qb, off, O.quantize(Qb, codebook, cfg.query_ma), X, dbc)[0]
        O.rank(S, cfg.topk)
        Sp = O.sif_scores_inverted(O.membership(S, cfg.sif_k1), card, entries)
        np.lexsort((np.arange(n_slice), -S, -Sp))[:cfg.topk]
        times.append(time.time() - t)
    return times


def slice_sample_text(cfg, n_slice, n_steps):
    return (f"{n_steps} steps of one query against a {n_slice:,}-shape slice ({n_slice / cfg.n_shapes:.1%} of the "
            f"{cfg.n_shapes:,} shapes) through the FP64 oracle: quantiser, Eq. 4 literally over the slice (its "
            f"database codes computed beforehand, untimed), top-{cfg.topk}, S-IF re-rank (Eqs. 13-14) over a seeded "
            f"stand-in activation of the slice; time per query = step time x {cfg.n_shapes / n_slice:.0f}")


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


# ---------------------------------------------------------------- reference arm
def reference_arm(cfg, args, rank):
    """``--impl reference``: the FP64 oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    cores = blas_threads()
    if cfg.generator == "counter":
        from synth import config_codebook
        n_slice = 1000
        cb = config_codebook(cfg)
        times = cpu_oracle_slice(cfg, args.warmup + args.steps, cb, n_slice)
        t = np.asarray(times[args.warmup:]) * (cfg.n_shapes / n_slice)
        sample = slice_sample_text(cfg, n_slice, args.steps)
    else:
        data = make_inputs(cfg, n_queries=max(8, args.steps + args.warmup))
        times, _ = cpu_oracle_run(cfg, data, 1, args.warmup + args.steps)
        t = np.asarray(times[args.warmup:])
        sample = "1 query per step through the FP64 oracle: Eq. 4 over all shapes, top-k, dense Eq. 8 re-rank " \
                 "(off-line database codes untimed; S-IF activations a seeded stand-in)"
    qps = len(t) / float(t.sum())
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(t.mean()),
            "p99_ms": 1e3 * float(np.percentile(t, 99)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg.name, "queries_per_step": 1, "db_shapes": cfg.n_shapes,
                       "views": cfg.n_views, "dim": cfg.dim, "codewords": cfg.n_codewords, "query_ma": cfg.query_ma,
                       "topk": cfg.topk, "sif_k1": cfg.sif_k1},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "cpu": cpu_model(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def make_inputs(cfg, n_queries=None):
    from synth import make_config_inputs
    return make_config_inputs(cfg, n_queries=n_queries)


# ---------------------------------------------------------------- one workload on the GPU
def measure_workload(cfg, args, gift, torch, dev, rank, world, codebook=None, serve_seconds=0.0,
                     recall_queries=None, keep_exact=True):
    """Index a workload, time its query steps (device and end to end), the exact path and
    optionally a serving session; returns (result dict, data, index still open)."""
    large = cfg.generator == "counter"
    R = cfg.rescore_r if args.rescore is None else args.rescore
    B = cfg.batch or cfg.n_queries
    t0 = time.time()
    build_s = None
    data = None
    if large:
        # database views drawn on the device chunk by chunk, three times (one per build pass)
        from synth import config_views
        ix = gift.Index.streamed(lambda f, n: config_views(cfg, f, n, device=dev),
                                 torch.from_numpy(codebook).to(dev), cfg.n_shapes, cfg.n_views, cfg.n_codewords,
                                 chunk_shapes=512, storage=cfg.storage, query_ma=cfg.query_ma, sif_k1=cfg.sif_k1,
                                 rescore_r=R)
        torch.cuda.synchronize()
        build_s = time.time() - t0
        log(f"[bench] {cfg.name}: streamed index built in {build_s:.1f}s: {ix.info()} "
            f"free {torch.cuda.mem_get_info(dev)[0] / 2**30:.1f} GiB")
        q_all = config_views(cfg, 0, cfg.n_queries, device=dev, query=True).view(-1, cfg.dim)
        qoff = np.arange(cfg.n_queries + 1, dtype=np.int64) * cfg.n_views
    else:
        data = make_inputs(cfg)
        if rank > 0:  # every rank serves its own query stream
            from synth.workload import query_views
            q, qo, _ = query_views(cfg.n_queries, cfg.query_views, cfg.dim, cfg.n_classes,
                                   cfg.query_seed + 100 * rank, cfg.centre_seed, cfg.noise, max_views=cfg.n_views)
            data["q"], data["q_off"] = q, qo
        log(f"[bench] {cfg.name}: inputs generated in {time.time() - t0:.1f}s")
        t0 = time.time()
        db_dev = torch.from_numpy(data["db"]).to(dev)
        ix = gift.Index(db_dev, torch.from_numpy(data["codebook"]).to(dev), cfg.n_shapes, cfg.n_views,
                        cfg.n_codewords, storage=cfg.storage, query_ma=cfg.query_ma, sif_k1=cfg.sif_k1,
                        rescore_r=R, keep_exact=keep_exact and not args.profile)
        torch.cuda.synchronize()
        build_s = time.time() - t0
        del db_dev
        log(f"[bench] {cfg.name}: index built in {build_s:.1f}s: {ix.info()}")
        q_all = torch.from_numpy(data["q"]).to(dev)
        qoff = np.asarray(data["q_off"], np.int64)
    nb = (len(qoff) - 1) // B
    first = (5 * rank) % nb  # ranks start at different batches of the query set
    batches = []
    for j in range(nb):
        i = (first + j) % nb
        lo, hi = qoff[i * B], qoff[(i + 1) * B]
        batches.append((q_all[lo:hi], (qoff[i * B:(i + 1) * B + 1] - lo).astype(np.int32)))
    topk, k1 = cfg.topk, cfg.sif_k1
    stream = torch.cuda.current_stream()
    out_q = (torch.empty((B, topk), dtype=torch.int32, device=dev), torch.empty((B, topk), device=dev))
    out_r = (torch.empty((B, topk), dtype=torch.int32, device=dev), torch.empty((B, topk), device=dev))

    def step(i, timing=False):
        qb, ob = batches[i % nb]
        ix.query(qb, ob, mode="fif", topk=topk, out=out_q)
        st_q = ix.timing() if timing else None
        ix.rerank(out_q[0], out_q[1], k1=k1, topk=topk, out=out_r)
        st_r = ix.timing() if timing else None
        return st_q, st_r

    # ---- device-timed steps (inputs resident in HBM; list stores larger than L2)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index) if not args.profile else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.nvtx.range_push("timed_steps")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    n_launch0 = gift.launch_count()
    ev[0].record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    n_launches = gift.launch_count() - n_launch0
    if args.profile:
        torch.cuda.nvtx.range_pop()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    t_tensor = torch.tensor([total_ms], device=dev)
    if world > 1:
        torch.distributed.all_reduce(t_tensor, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
    total_ms = float(t_tensor.item())
    if args.profile:
        # one more step, timed by the library, outside the captured range: the work
        # counters that scale an ncu capture of these launches to other workloads
        # (the batch of the first timed step; a capture of one step, or of a
        # workload with a single batch, matches them exactly)
        ix.set_timing(True)
        st_q, _ = step(args.warmup, timing=True)
        ix.set_timing(False)
        eb = 1 if cfg.storage == "fp8" else (2 if cfg.storage == "bf16" else 4)
        counters = {k: st_q[k] for k in ("scan_bytes", "rescore_bytes", "scan_pairs", "assign_rows", "rescore_items",
                                         "rescore_items_kept", "cand_pairs", "cand_rows", "rescore_rows_read")}
        counters["touched_rows"] = st_q["scan_bytes"] / (cfg.dim * eb + 12)
        log(f"[bench] profile run: {total_ms / args.steps:.3f} ms/step; work per step {json.dumps(counters)}")
        return {"ms_per_step": total_ms / args.steps, "work": counters}, data, ix

    # ---- per-stage device times (CUDA events recorded by the library on this stream)
    ix.set_timing(True)
    stages = [step(i, timing=True) for i in range(max(3, min(args.steps, 10)))]
    ix.set_timing(False)
    clocks = sampler.stop()

    def avg(key, which=0):
        return statistics.mean(s_[which][key] for s_ in stages)

    st = {k: avg(k) for k in ("assign_ms", "bucket_ms", "scan_ms", "combine_ms", "topk_ms", "rescore_ms",
                               "total_ms", "assign_kernel_ms", "scan_kernel_ms", "rescore_kernel_ms")}
    st["rerank_ms"] = avg("rerank_ms", 1)
    work = {k: stages[-1][0][k] for k in ("scan_bytes", "rescore_bytes", "scan_pairs", "assign_rows")}
    cand = {k: stages[-1][0][k] for k in ("rescore_items", "rescore_items_kept", "cand_pairs", "cand_rows",
                                          "rescore_rows_read")}

    # ---- device time per step at other rescore depths (recall at each depth comes from the oracle)
    depth_sweep = None
    if large and R > 0:
        depth_sweep = {}
        for r_ in (0, 200, 400, 600, 800, R):
            if r_ > R or (0 < r_ < topk):
                continue
            ix.set_rescore_depth(r_)
            step(0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(5):
                step(i)
            e1.record(stream)
            torch.cuda.synchronize()
            depth_sweep[r_] = {"ms_per_step": e0.elapsed_time(e1) / 5,
                               "queries_per_s": 5 * B / (e0.elapsed_time(e1) / 1e3)}
        ix.set_rescore_depth(R)

    # ---- end to end through the C ABI with host buffers: pinned query features in,
    # ids / scores out, every step; three streams rotate so that the copies of
    # one batch overlap the kernels of the others
    q_host = [(batches[i][0].cpu().pin_memory(), batches[i][1]) for i in range(min(nb, 8))]
    n_streams = 3
    streams = [torch.cuda.Stream(device=dev) for _ in range(n_streams)]
    hq = [(torch.empty((B, topk), dtype=torch.int32).pin_memory(), torch.empty((B, topk)).pin_memory())
          for _ in range(n_streams)]
    hr = [(torch.empty((B, topk), dtype=torch.int32).pin_memory(), torch.empty((B, topk)).pin_memory())
          for _ in range(n_streams)]

    def e2e_step(i):
        j = i % n_streams
        qh, ob = q_host[i % len(q_host)]
        streams[j].synchronize()  # this stream's host buffers are free again
        ix.query(qh, ob, mode="fif", topk=topk, out=hq[j], stream=streams[j])
        ix.rerank(hq[j][0], hq[j][1], k1=k1, topk=topk, out=hr[j], stream=streams[j])

    for i in range(args.warmup):
        e2e_step(i)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter()
    for i in range(args.steps):
        e2e_step(i)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t_e2e) * 1e3 / args.steps
    h2d = q_host[0][0].numel() * 4 + 2 * B * topk * 4
    d2h = 4 * B * topk * 4
    del q_host

    # ---- exact match (Eq. 3, FP32-level) on a sub-batch, the plain path, with its own clocks
    nx = 16 if large else min(B, 64)
    qx, ox = batches[0][0][:int(batches[0][1][nx])], batches[0][1][:nx + 1]
    ix.query(qx[:int(ox[1])], ox[:2], mode="exact", topk=topk)
    torch.cuda.synchronize()
    reps = 3
    x_sampler = ClockSampler(dev.index)
    x_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    x_ev[0].record(stream)
    for _ in range(reps):
        ix.query(qx, ox, mode="exact", topk=topk)
    x_ev[1].record(stream)
    torch.cuda.synchronize()
    exact_ms = x_ev[0].elapsed_time(x_ev[1]) / reps
    exact = {"value": nx / (exact_ms / 1e3), "unit": "queries/s", "queries": nx, "ms": exact_ms,
             "clocks": x_sampler.stop(),
             "source": ("list-ordered two-part BF16 store (FP32-level), every database view" if large else
                        "shape-ordered two-part BF16 copy (FP32-level), every database view")}

    # ---- GPU results of the sampled recall queries at several rescore depths (compared on the host later)
    recall_gpu = None
    if recall_queries is not None:
        from synth import config_views
        qs = torch.cat([config_views(cfg, b, 1, device=dev, query=True)[0] for b in recall_queries])
        off_s = (np.arange(len(recall_queries) + 1) * cfg.n_views).astype(np.int32)
        ids, sc = ix.query(qs, off_s, mode="fif", topk=topk)
        recall_gpu = {"ids": ids.cpu().numpy(), "scores": sc.cpu().numpy(), "sweep": {}}
        for r_ in (0, 100, 200, 400, 600, 800, R):
            if r_ > R or (0 < r_ < topk):
                continue
            ix.set_rescore_depth(r_)
            recall_gpu["sweep"][r_] = ix.query(qs, off_s, mode="fif", topk=topk)[0].cpu().numpy()
        ix.set_rescore_depth(R)
        del qs

    # ---- serving: Poisson arrivals, view counts uniform in {12, 20, 64}, continuous batching
    serving = None
    if serve_seconds > 0 and rank == 0:
        pool = np.concatenate([batches[i][0][:int(batches[i][1][-1])].cpu().numpy() for i in range(min(nb, 4))])
        del batches, q_all
        batches = None
        torch.cuda.empty_cache()  # the server's scratch is admitted by free memory
        serving = run_serving(gift, ix, cfg, pool, serve_seconds, args.serve_rate, topk)
        log(f"[bench] serving: {serving}")

    value = world * args.steps * B / (total_ms / 1e3)
    res = {"value": value, "ms_per_step": total_ms / args.steps,
           "p50_ms": float(np.percentile(per_step, 50)), "p99_ms": float(np.percentile(per_step, 99)),
           "step_ms": [round(float(x), 3) for x in per_step],
           "config": {"workload": cfg.name, "db_shapes": cfg.n_shapes, "views": cfg.n_views, "dim": cfg.dim,
                      "codewords": cfg.n_codewords, "query_ma": cfg.query_ma, "queries_per_step": B,
                      "storage": cfg.storage, "rescore_r": R, "topk": topk, "sif_k1": k1,
                      "l2": "inputs larger than L2 (list store " + ("52 GB" if large else "6.3 GB") + ")",
                      "parallelism": f"replica x{world}"},
           "exact": dict(exact, speedup_fif_over_exact=value / world / exact["value"]),
           "stages_ms": st,
           "e2e": {"value": B / (e2e_ms / 1e3) * world, "unit": "queries/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "streams": n_streams},
           "clocks": clocks, "gpu_launches": n_launches, "gpu_launches_per_step": n_launches / args.steps,
           "build_s": build_s, "serving": serving, "rescore_depth_sweep": depth_sweep}
    peaks, peak_src = measured_peaks()
    res["roofline"] = roofline(cfg, st, work["scan_pairs"], work["scan_bytes"], work["rescore_bytes"],
                               work["assign_rows"], peaks, peak_src, cand=cand)
    res["_recall_gpu"] = recall_gpu
    res["_batches"] = batches
    return res, data, ix


def run_serving(gift, ix, cfg, pool, seconds, rate, topk):
    import threading
    sv = gift.Server(ix, slots=3, max_batch_queries=256, max_batch_views=256 * 64, topk=topk, rerank=True)
    g = np.random.default_rng(5000 + cfg.seed)
    n_req = max(1, int(rate * seconds))
    vcounts = g.choice(np.array([12, 20, 64]), size=n_req)
    gaps = g.exponential(1.0 / rate, size=n_req)
    pool_off = np.arange(len(pool) // cfg.n_views + 1) * cfg.n_views
    nq_pool = len(pool_off) - 1
    tickets = [None] * n_req

    def producer():
        t = time.perf_counter()
        for i in range(n_req):
            t += gaps[i]
            while time.perf_counter() < t:
                pass
            b = i % nq_pool
            tickets[i] = sv.submit(pool[pool_off[b]:pool_off[b] + int(vcounts[i])])

    t_s = time.perf_counter()
    th = threading.Thread(target=producer)
    th.start()
    done = 0
    while done < n_req:
        while tickets[done] is None:
            time.sleep(1e-4)
        sv.wait(tickets[done], timeout_ms=120000)
        done += 1
    th.join()
    wall = time.perf_counter() - t_s
    sst = sv.stats()
    sv.close()
    return {"arrival_rate": rate, "seconds": seconds, "requests": n_req, "view_counts": [12, 20, 64],
            "queries_per_s": n_req / wall, "p50_ms": sst["p50_ms"], "p99_ms": sst["p99_ms"], "max_ms": sst["max_ms"],
            "batches": sst["batches"], "mean_batch": sst["mean_batch"], "slots": 3, "index": cfg.name,
            "result": f"top-{topk} after S-IF re-rank"}


def dense_recall(cfg, data, ix, res, topk):
    """recall@topk of the workload's first batch on 4 sampled queries against the FP64 oracle's
    Eq. 4 ranking (the oracle quantises every database view in float64)."""
    from oracle import gift_oracle as O
    t = time.time()
    N, Nv, D = cfg.n_shapes, cfg.n_views, cfg.dim
    db_codes = O.quantize(data["db"].reshape(-1, D), data["codebook"], 1).reshape(N, Nv)
    log(f"[bench] oracle database codes in {time.time() - t:.1f}s")
    B = cfg.batch or cfg.n_queries
    qoff = np.asarray(data["q_off"], np.int64)
    q0 = data["q"][:qoff[B]]
    ids, sc = ix.query(q0, (qoff[:B + 1]).astype(np.int32), mode="fif", topk=topk)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    rec, errs = [], []
    for b in (0, B // 3, (2 * B) // 3, B - 1):
        lo, hi = qoff[b], qoff[b + 1]
        Qb = data["q"][lo:hi]
        Sref = O.fif_scores(Qb, np.array([0, hi - lo]), O.quantize(Qb, data["codebook"], cfg.query_ma), data["db"],
                            db_codes)[0]
        ref_ids, _ = O.rank(Sref, topk)
        rec.append(len(set(ids[b].tolist()) & set(ref_ids.tolist())) / topk)
        errs.append(float(np.max(np.abs(sc[b] - Sref[ids[b]]) / np.maximum(np.abs(Sref[ids[b]]), 1e-30))))
    log(f"[bench] recall {rec} max rel err {max(errs):.2e} in {time.time() - t:.1f}s")
    return {"value": float(np.mean(rec)), "min": float(np.min(rec)), "queries": len(rec),
            "max_rel_score_err": float(np.max(errs)), "vs": "FP64 oracle, Eq. 4"}, db_codes


# ---------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gift", choices=["gift", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--second-config", default=SECOND_CONFIG,
                    help="a second workload measured after the first on rank 0 at N = 1 ('none' = skip)")
    ap.add_argument("--no-recall", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true", help="steps only (for ncu launch lists)")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="serving session length (default 15 s on the first workload; 0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation measurement")
    ap.add_argument("--no-aca", action="store_true", help="skip the two-measure re-rank measurement")
    ap.add_argument("--no-kmeans", action="store_true", help="skip the GPU k-means measurement")
    ap.add_argument("--no-render", action="store_true", help="skip the projection front end measurement")
    ap.add_argument("--diff-only", action="store_true",
                    help="only the differentiation workload (forward + backward; for ncu launch lists)")
    ap.add_argument("--diff-shapes", type=int, default=None, help="override its database shapes (small ncu case)")
    ap.add_argument("--diff-queries", type=int, default=None, help="override its query shapes (small ncu case)")
    ap.add_argument("--rescore", type=int, default=None, help="override the config's rescore depth R")
    ap.add_argument("--batch", type=int, default=None,
                    help="override the config's queries per call (profiling cases of the timed workload's list mix)")
    ap.add_argument("--oracle-queries", type=int, default=8, help="sampled queries for recall (large configs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if not args.profile else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    from synth import CONFIGS
    cfg = CONFIGS[args.config]
    if args.batch:
        import dataclasses
        cfg = dataclasses.replace(cfg, batch=int(args.batch))
    if args.impl == "reference":
        reference_arm(cfg, args, rank)
        return

    large = cfg.generator == "counter"
    oracle_conn = oracle_proc = codebook = q_sample = None
    if large:
        from synth import config_codebook
        t0 = time.time()
        codebook = config_codebook(cfg)
        log(f"[bench] codebook fixture in {time.time() - t0:.1f}s")
        q_sample = sorted({int(round(x)) for x in np.linspace(0, cfg.n_queries - 1, max(1, args.oracle_queries))})
        if not args.no_recall and not args.profile and rank == 0 and world == 1:  # recall: the N = 1 run
            import multiprocessing as mp
            ctx = mp.get_context("spawn")  # before the first CUDA call
            oracle_conn, child = ctx.Pipe(duplex=False)
            threads = max(1, (os.cpu_count() or 4) - 4)  # leave cores for the launch and serving threads
            saved = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
            for v in saved:
                os.environ[v] = str(threads)
            oracle_proc = ctx.Process(target=oracle_bounded_worker,
                                      args=(cfg.name, q_sample, codebook, cfg.topk, threads, child), daemon=True)
            oracle_proc.start()
            for v, old_v in saved.items():
                if old_v is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old_v

    import torch
    import paper_1604_01879_gb300 as gift
    from paper_1604_01879_gb300 import build as gbuild

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        gbuild.build()
    if world > 1:
        torch.distributed.barrier()
    gift.load()
    if args.diff_only:
        if rank == 0:
            print(json.dumps({"differentiation": bench_differentiation(
                gift, torch, dev, torch.cuda.current_stream(), reps=max(1, args.steps), n_shapes=args.diff_shapes,
                n_queries=args.diff_queries)}))
        return

    serve_s = (15.0 if large else 5.0) if args.serve_seconds is None else args.serve_seconds
    if world > 1:
        serve_s = 0.0  # serving is measured on one GPU
    res, data, ix = measure_workload(cfg, args, gift, torch, dev, rank, world, codebook=codebook,
                                     serve_seconds=serve_s,
                                     recall_queries=q_sample if oracle_conn is not None else None)
    if args.profile:
        ix.close()
        return
    recall_gpu = res.pop("_recall_gpu")
    res.pop("_batches")
    value = res["value"]
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "p50_ms": res["p50_ms"], "p99_ms": res["p99_ms"],
            "step_ms": res["step_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "e4m3" if cfg.storage == "fp8" else "bf16", "data": "synthetic", "config": res["config"],
            "exact": res["exact"], "stages_ms": res["stages_ms"], "e2e": res["e2e"], "clocks": res["clocks"],
            "gpu_launches": res["gpu_launches"], "gpu_launches_per_step": res["gpu_launches_per_step"],
            "build_s": res["build_s"], "serving": res["serving"], "roofline": res["roofline"],
            "rescore_depth_sweep": res["rescore_depth_sweep"]}
    db_codes = None
    if not large and not args.no_recall and rank == 0:
        line["recall_at_100"], db_codes = dense_recall(cfg, data, ix, res, cfg.topk)
    if not large and not args.no_cpu_baseline and rank == 0 and world == 1:
        times, _ = cpu_oracle_run(cfg, data, 1, 4, db_codes=db_codes)
        line["cpu_baseline"] = {"value": 1.0 / statistics.mean(times[1:]), "unit": "queries/s",
                                "cores": blas_threads(), "cpu": cpu_model(), "kind": "oracle",
                                "sample": f"3 queries (after 1 warm-up) through the FP64 oracle: Eq. 4 over all "
                                          f"{cfg.n_shapes:,} shapes, top-{cfg.topk}, dense Eq. 8 re-rank over "
                                          f"{cfg.n_shapes:,} shapes (the database activations a seeded stand-in "
                                          f"for timing: dense Eq. 8 costs the same whatever their values)"}
    ix.close()
    del ix
    torch.cuda.empty_cache()

    # ---- a second workload (rank 0, N = 1): the ModelNet40-sized index and the measurements
    # that use its inputs (two measures, k-means, rendering, differentiation)
    if rank == 0 and world == 1 and args.second_config != "none":
        cfg2 = CONFIGS[args.second_config]
        a2 = argparse.Namespace(**vars(args))
        res2, data2, ix2 = measure_workload(cfg2, a2, gift, torch, dev, rank, world, serve_seconds=0.0)
        batches2 = res2.pop("_batches")
        res2.pop("_recall_gpu")
        second = {k: res2[k] for k in ("value", "ms_per_step", "p50_ms", "p99_ms", "config", "exact", "e2e",
                                       "roofline", "stages_ms", "clocks", "gpu_launches_per_step", "build_s")}
        second["unit"] = "queries/s"
        stream = torch.cuda.current_stream()
        if not args.no_aca and cfg2.sif_k1 > 0 and data2 is not None:
            second["two_measure_rerank"] = bench_aca(cfg2, gift, torch, dev, stream, ix2, batches2, cfg2.topk,
                                                     cfg2.rescore_r)
        ix2.close()
        del ix2, batches2
        torch.cuda.empty_cache()
        line["second_workload"] = second
        if not args.no_kmeans and data2 is not None:
            line["kmeans"] = bench_kmeans(cfg2, gift, torch, dev, stream, data2)
        if not args.no_render:
            line["rendering"] = bench_render(gift, torch, dev, stream)
        if not args.no_diff:
            line["differentiation"] = bench_differentiation(gift, torch, dev, stream)
        log(f"[bench] second workload: {second}")

    # ---- recall@100 vs the FP64 oracle on sampled queries (large config: bounded oracle process)
    if large and oracle_conn is not None:
        log("[bench] waiting for the oracle process")
        got = oracle_conn.recv() if oracle_conn.poll(3600) else {"error": "oracle timed out"}
        oracle_proc.join(timeout=60)
        if "error" in got:
            line["recall_at_100"] = {"value": None, "error": got["error"]}
        else:
            topk = cfg.topk
            ids, sc = recall_gpu["ids"], recall_gpu["scores"]
            rec, errs = [], []
            for j in range(len(q_sample)):
                ref_ids = got["ids"][j]
                rec.append(len(set(ids[j].tolist()) & set(ref_ids)) / topk)
                ref = dict(zip(ref_ids, got["scores"][j]))
                errs += [abs(float(s_) - ref[int(p_)]) / max(abs(ref[int(p_)]), 1e-30)
                         for p_, s_ in zip(ids[j], sc[j]) if int(p_) in ref]
            sweep = {r_: float(np.mean([len(set(v[j].tolist()) & set(got["ids"][j])) / topk
                                        for j in range(len(q_sample))]))
                     for r_, v in recall_gpu["sweep"].items()}
            line["recall_at_100"] = {"value": float(np.mean(rec)), "min": float(np.min(rec)),
                                     "queries": len(rec), "query_ids": q_sample,
                                     "max_rel_score_err": float(np.max(errs)) if errs else None,
                                     "vs": "FP64 oracle, Eq. 4 (top-k pruned by the Eq. 3 bound)",
                                     "oracle_shapes_visited": got["visited"],
                                     "oracle_seconds_per_query": got["seconds"] / len(q_sample),
                                     "vs_rescore_depth": sweep}
        log(f"[bench] recall: {line['recall_at_100']}")

    # ---- CPU baseline of the large config: the oracle on a bounded slice (rank 0, N = 1),
    # after the oracle process has finished so the two do not share the cores
    if large and not args.no_cpu_baseline and rank == 0 and world == 1:
        n_slice, n_steps = 1000, 4
        times = cpu_oracle_slice(cfg, n_steps + 1, codebook, n_slice)
        t = np.asarray(times[1:]) * (cfg.n_shapes / n_slice)
        line["cpu_baseline"] = {"value": len(t) / float(t.sum()), "unit": "queries/s", "cores": blas_threads(),
                                "cpu": cpu_model(), "kind": "oracle",
                                "sample": slice_sample_text(cfg, n_slice, n_steps) + " (after 1 warm-up step)"}

    if rank == 0:
        print(json.dumps(line))


def bench_aca(cfg, gift, torch, dev, stream, ix1, batches, topk, R, reps=5):
    """The paper's default re-ranking: a second measure's index (synthetic stand-in for a
    second CNN layer), co-augmented activations (Eq. 11, k2 = 4) fused by Eq. 9 (alpha = 0.5),
    S' through their own inverted file. Step = query on both indices + the fused re-rank."""
    from synth import make_config_inputs, second_measure
    c2 = second_measure(cfg)
    t0 = time.time()
    d2 = make_config_inputs(c2)
    ix2 = gift.Index(torch.from_numpy(d2["db"]).to(dev), torch.from_numpy(d2["codebook"]).to(dev), c2.n_shapes,
                     c2.n_views, c2.n_codewords, storage=c2.storage, query_ma=c2.query_ma, sif_k1=c2.sif_k1,
                     rescore_r=R, keep_exact=False)
    torch.cuda.synchronize()
    t_ix2 = time.time() - t0
    t0 = time.time()
    aca = gift.Aca(ix1, ix2, k2=4, alpha=0.5, mode="co")
    torch.cuda.synchronize()
    t_aca = time.time() - t0
    pairs = int(aca.export()[0][-1])
    q2 = torch.from_numpy(d2["q"]).to(dev)
    B = batches[0][1].shape[0] - 1
    qoff2 = np.asarray(d2["q_off"], np.int64)
    b2 = [(q2[qoff2[i * B]:qoff2[(i + 1) * B]], (qoff2[i * B:(i + 1) * B + 1] - qoff2[i * B]).astype(np.int32))
          for i in range((len(qoff2) - 1) // B)]
    nb = min(len(batches), len(b2))

    def step(i):
        c1 = ix1.query(*batches[i % nb], mode="fif", topk=topk)
        c2_ = ix2.query(*b2[i % nb], mode="fif", topk=topk)
        e[1].record(stream)
        return aca.rerank(c1, c2_, topk=topk)

    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    step(0)
    torch.cuda.synchronize()
    tot, rr = [], []
    for i in range(reps):
        e[0].record(stream)
        step(i)
        e[2].record(stream)
        torch.cuda.synchronize()
        tot.append(e[0].elapsed_time(e[2]))
        rr.append(e[1].elapsed_time(e[2]))
    aca.close()
    ix2.close()
    del q2
    torch.cuda.empty_cache()
    t_ms, r_ms = statistics.median(tot), statistics.median(rr)
    return {"measure2": c2.name, "k1": cfg.sif_k1, "k2": 4, "alpha": 0.5, "mode": "co-augmentation (Eq. 11)",
            "queries_per_step": B, "step_ms": t_ms, "queries_per_s": B / (t_ms / 1e3), "fused_rerank_ms": r_ms,
            "fused_sif_pairs": pairs, "build_index2_s": t_ix2, "build_fused_sif_s": t_aca}


def bench_render(gift, torch, dev, stream, n_meshes=256, reps=3):
    """Depth-buffer views (Sec. 2.1) of a batch of seeded meshes: 8 azimuths x 8 elevations
    at 224 x 224, device inputs, device-timed."""
    from synth.meshes import mesh_batch
    V, T, vo, to = mesh_batch(0, n_meshes, 40, 61)
    Vd, Td = torch.from_numpy(V).to(dev), torch.from_numpy(T).to(dev)
    out = torch.empty((n_meshes, 64, 224, 224), dtype=torch.float32, device=dev)
    gift.render_views(Vd, Td, vo, to, 8, 8, 224, 224, out=out)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    for _ in range(reps):
        gift.render_views(Vd, Td, vo, to, 8, 8, 224, 224, out=out)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / reps
    covered = float((out < 2).float().mean().item())
    del out, Vd, Td
    torch.cuda.empty_cache()
    return {"meshes": n_meshes, "triangles_per_mesh": int(to[1] - to[0]), "views": 64, "image": [224, 224],
            "ms": ms, "ms_per_mesh": ms / n_meshes, "meshes_per_s": n_meshes / (ms / 1e3),
            "covered_pixel_fraction": covered, "output_gb": n_meshes * 64 * 224 * 224 * 4 / 1e9}


def bench_kmeans(cfg, gift, torch, dev, stream, data):
    """GPU Lloyd k-means on the codebook fixture's sample (its rows, K, iterations and initial rows),
    device-timed; the host fixture (numpy, FP32 distances) is timed on one iteration for context."""
    from synth import codebook_sample_shapes, kmeans_init_rows, kmeans_codebook
    X = np.ascontiguousarray(data["db"][codebook_sample_shapes(cfg)].reshape(-1, cfg.dim))
    init = kmeans_init_rows(len(X), cfg.n_codewords, cfg.codebook_seed)
    Xd = torch.from_numpy(X).to(dev)
    gift.kmeans(Xd, init, iters=1)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    gift.kmeans(Xd, init, iters=cfg.kmeans_iters)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1])
    t0 = time.time()
    kmeans_codebook(X, cfg.n_codewords, cfg.codebook_seed, 1)
    host_it = time.time() - t0
    del Xd
    torch.cuda.empty_cache()
    return {"rows": len(X), "dim": cfg.dim, "K": cfg.n_codewords, "iters": cfg.kmeans_iters, "gpu_ms": ms,
            "gpu_ms_per_iter": ms / max(1, cfg.kmeans_iters), "host_fixture_s_per_iter": host_it,
            "note": "exact assignment (tensor-core quantiser) + two-float FP32 means; the host fixture uses FP32 distances"}


def bench_differentiation(gift, torch, dev, stream, reps=3, n_shapes=None, n_queries=None):
    """Forward + backward of the projected match (Eq. 3 after u = W q) on the
    differentiation workload (or a smaller one of the same recipe); device-timed
    with CUDA events."""
    from synth import DIFF_WORKLOAD as W_, shape_views, projection_matrix, upstream_grad
    nq, N, nv, D, dout = W_["n_queries"], W_["n_shapes"], W_["n_views"], W_["dim"], W_["d_out"]
    nq, N = n_queries or nq, n_shapes or N
    s = W_["seed"]
    q = torch.from_numpy(shape_views(0, nq, nv, D, W_["n_classes"], 2000 + s, 4000 + s)).to(dev).to(
        torch.bfloat16).reshape(nq * nv, D)
    p = torch.from_numpy(shape_views(0, N, nv, D, W_["n_classes"], 1000 + s, 4000 + s)).to(dev).to(torch.bfloat16)
    W = torch.from_numpy(projection_matrix(dout, D, 3000 + s, W_["w_std"])).to(dev).to(torch.bfloat16)
    G = torch.from_numpy(upstream_grad(nq, N, 5000 + s)).to(dev)
    off = np.arange(0, nq * nv + 1, nv, dtype=np.int32)
    S, am = gift.match_forward(q, off, p, W)
    gift.match_backward(q, off, p, W, G, am)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fw, bw = [], []
    for _ in range(reps):
        e[0].record(stream)
        S, am = gift.match_forward(q, off, p, W)
        e[1].record(stream)
        gift.match_backward(q, off, p, W, G, am)
        e[2].record(stream)
        torch.cuda.synchronize()
        fw.append(e[0].elapsed_time(e[1]))
        bw.append(e[1].elapsed_time(e[2]))
    nr = N * nv
    proj = 2.0 * (nq * nv + nr) * D * dout
    sim = 2.0 * (nq * nv) * nr * dout
    f_ms, b_ms = statistics.median(fw), statistics.median(bw)
    name = W_["name"] if (nq, N) == (W_["n_queries"], W_["n_shapes"]) else f"match{nq}x{N}x{nv}_d{D}_p{dout}_bf16"
    out = {"workload": name, "forward_ms": f_ms, "backward_ms": b_ms,
           "useful_tflop_fwd": (proj + sim) / 1e12, "useful_tflop_bwd": (proj + 2 * proj) / 1e12,
           "fwd_useful_tflops": (proj + sim) / (f_ms / 1e3) / 1e12,
           "bwd_useful_tflops": 3 * proj / (b_ms / 1e3) / 1e12,
           "note": "similarity and dW/dQ/dP GEMMs run two-part BF16 (3 products); projections of BF16 inputs 1 product; "
                    "the one-hot gradient products are FP32 gathers on the CUDA cores"}
    del q, p, W, G, S, am
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
