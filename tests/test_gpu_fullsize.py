"""Full-size parity on sampled outputs, in the launch configuration bench.py times.

ModelNet40-sized index (12,000 shapes x 64 views x D=4096, K=1024, BF16 store,
FP32 rescore of the top 200, S-IF k1=50) queried with one 1,000-query batch:
sampled codes, the full top-100 of sampled queries against the oracle's Eq. 4
ranking (the oracle quantises all 768,000 database views in float64), S-IF
entries and S' of sampled shapes. Differentiation workload (256 x 64 query
views against 4,096 x 64 database views, D=4096 BF16, projection to 512):
S, argmax and dQ of sampled query views against the oracle.
"""
import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import CONFIGS, make_config_inputs, DIFF_WORKLOAD, shape_views, projection_matrix, upstream_grad
from tests.parity import (FIX, RTOL, ErrorBand, assert_codes, assert_topk, close, code_margins, recall,
                          reference_memberships)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2(gpu_lib):
    import torch
    cfg = CONFIGS["db12000x64_d4096_k1024"]
    d = make_config_inputs(cfg)
    N, Nv, D, K = cfg.n_shapes, cfg.n_views, cfg.dim, cfg.n_codewords
    ix = gpu_lib.Index(torch.from_numpy(d["db"]).cuda(), torch.from_numpy(d["codebook"]).cuda(), N, Nv, K,
                       storage=cfg.storage, query_ma=cfg.query_ma, sif_k1=cfg.sif_k1, rescore_r=cfg.rescore_r,
                       keep_exact=False)
    q = torch.from_numpy(d["q"]).cuda()
    ids, sc = ix.query(q, d["q_off"], mode="fif", topk=cfg.topk)
    torch.cuda.synchronize()
    db_codes = O.quantize(d["db"].reshape(-1, D), d["codebook"], 1).reshape(N, Nv)
    yield dict(cfg=cfg, d=d, ix=ix, ids=ids.cpu().numpy(), sc=sc.cpu().numpy(), q=q, db_codes=db_codes)
    ix.close()


def _oracle_row(c, Qb):
    off = np.array([0, len(Qb)])
    qc = O.quantize(Qb, c["d"]["codebook"], c["cfg"].query_ma)
    return O.fif_scores(Qb, off, qc, c["d"]["db"], c["db_codes"])[0]


def test_sampled_codes(c2):
    import torch
    cfg, d = c2["cfg"], c2["d"]
    codes, off, rows = c2["ix"].export_fif()
    g = np.random.default_rng(0)
    pick = g.choice(cfg.n_shapes * cfg.n_views, 3000, replace=False)
    X = d["db"].reshape(-1, cfg.dim)
    assert_codes(codes[pick].reshape(-1, 1), c2["db_codes"].reshape(-1)[pick].reshape(-1, 1),
                 code_margins(X[pick], d["codebook"], 1))
    qp = g.choice(len(d["q"]), 2000, replace=False)
    qcodes = c2["ix"].assign(torch.from_numpy(d["q"][qp]).cuda(), 1).cpu().numpy()
    assert_codes(qcodes, O.quantize(d["q"][qp], d["codebook"], 1), code_margins(d["q"][qp], d["codebook"], 1))
    assert off[-1] == cfg.n_shapes * cfg.n_views


def test_sampled_queries_top100_and_recall(c2):
    d, cfg = c2["d"], c2["cfg"]
    qoff = d["q_off"]
    rec = []
    for b in (0, 333, 999):
        ref = _oracle_row(c2, d["q"][qoff[b]:qoff[b + 1]])
        assert_topk(c2["ids"][b], c2["sc"][b], ref, cfg.topk)
        rec.append(recall(c2["ids"][b], ref, cfg.topk))
    assert min(rec) >= 0.99


def test_sampled_sif_entries_and_rerank(c2):
    """S-IF entries of sampled shapes and S' of one query's re-ranked top-5 against the oracle:
    memberships within the score tolerance (plus half a fixed-point step), S' within the bound
    propagated from the memberships' FP32 error (tests/parity.py); the oracle's memberships are
    taken on the GPU's neighbour sets once those are checked to be correct first-k1 sets."""
    import torch
    d, cfg = c2["d"], c2["cfg"]
    N, Nv, k1 = cfg.n_shapes, cfg.n_views, cfg.sif_k1
    off, ids, mem, card = c2["ix"].export_sif()
    X = d["db"]
    rows = {}

    def gpu_row(p):  # N_k1(p) and F_p from the exported entries
        if p not in rows:
            F, members = np.zeros(N), []
            for i in range(N):
                seg = ids[off[i]:off[i + 1]]
                j = np.searchsorted(seg, p)
                if j < len(seg) and seg[j] == p:
                    members.append(i)
                    F[i] = mem[off[i] + j] * FIX
            rows[p] = (np.asarray(members), F)
        return rows[p]

    def ref_row(p):  # oracle memberships of database shape p on the GPU's neighbour set
        return reference_memberships(_oracle_row(c2, X[p]), gpu_row(p)[0], k1)

    band = ErrorBand()
    for p in (5, 6789):
        F_ref, (members, F) = ref_row(p), gpu_row(p)
        assert close(F, F_ref, RTOL, FIX / 2).all()
        assert abs(card[p] * FIX - F_ref.sum()) <= RTOL * F_ref.sum() + k1 * FIX / 2
        band.add(F, F_ref)
    # S' of the re-ranked top-5 of one query
    b = 0
    qoff = d["q_off"]
    rid, rsp = c2["ix"].rerank(torch.from_numpy(c2["ids"][:1]).cuda(), torch.from_numpy(c2["sc"][:1]).cuda(),
                               k1=k1, topk=5)
    rid, rsp = rid.cpu().numpy()[0], rsp.cpu().numpy()[0]
    Fq = reference_memberships(_oracle_row(c2, d["q"][qoff[b]:qoff[b + 1]]), c2["ids"][b, :k1], k1)
    gq = np.zeros(N)
    gq[c2["ids"][b, :k1]] = c2["sc"][b, :k1]
    band.add(gq, Fq)
    refs = {}
    for p in rid:
        refs[int(p)] = ref_row(int(p))
        band.add(gpu_row(int(p))[1], refs[int(p)])
    rtol, atol = band.sprime_tolerance(k1, Fq.sum())
    assert rtol <= 1e-5, (band.lo, band.hi)
    for p, v in zip(rid, rsp):
        ref = O.contextual(Fq, refs[int(p)])
        assert abs(v - ref) <= rtol * ref + atol, (p, v, ref)


DIFF_SAMPLED_SHAPES = (5, 3001)


@pytest.fixture(scope="module")
def diff(gpu_lib):
    import torch
    W_ = DIFF_WORKLOAD
    nq, N, nv, D, dout, s = W_["n_queries"], W_["n_shapes"], W_["n_views"], W_["dim"], W_["d_out"], W_["seed"]
    Q = shape_views(0, nq, nv, D, W_["n_classes"], 2000 + s, 4000 + s).reshape(nq * nv, D)
    P = shape_views(0, N, nv, D, W_["n_classes"], 1000 + s, 4000 + s)
    Wm = projection_matrix(dout, D, 3000 + s, W_["w_std"])
    G = upstream_grad(nq, N, 5000 + s)
    qb = torch.from_numpy(Q).cuda().to(torch.bfloat16)
    pb = torch.from_numpy(P).cuda().to(torch.bfloat16)
    wb = torch.from_numpy(Wm).cuda().to(torch.bfloat16)
    off = np.arange(0, nq * nv + 1, nv, dtype=np.int32)
    S, am = gpu_lib.match_forward(qb, off, pb, wb)
    dW, dQ, dP = gpu_lib.match_backward(qb, off, pb, wb, torch.from_numpy(G).cuda(), am, need=(False, True, True))
    p_rows = {p: dP[p].cpu().numpy() for p in DIFF_SAMPLED_SHAPES}  # [nv, D] of sampled database shapes
    del dP
    Qf, Pf, Wf = (t.float().cpu().numpy() for t in (qb, pb, wb))
    yield dict(S=S.cpu().numpy(), am=am.cpu().numpy(), dQ=dQ.cpu().numpy(), dP=p_rows, Q=Qf, P=Pf, W=Wf, G=G,
               nv=nv, N=N)


def test_differentiation_sampled_views(diff):
    Q, P, W, G, nv, N = diff["Q"], diff["P"], diff["W"], diff["G"], diff["nv"], diff["N"]
    V = P.reshape(-1, P.shape[2]).astype(np.float64) @ W.T.astype(np.float64)
    Vn = V / np.linalg.norm(V, axis=1, keepdims=True)
    for b in (3, 200):
        rows = np.arange(b * nv, (b + 1) * nv)
        U = Q[rows].astype(np.float64) @ W.T.astype(np.float64)
        Un = U / np.linalg.norm(U, axis=1, keepdims=True)
        s = (Un @ Vn.T).reshape(nv, N, nv)
        S = s.max(axis=2).mean(axis=0)
        assert np.allclose(diff["S"][b], S, rtol=1e-5, atol=1e-6)
        top2 = np.sort(s, axis=2)[:, :, -2:]
        clear = (top2[:, :, 1] - top2[:, :, 0]) > 1e-4
        assert np.array_equal(diff["am"][rows][clear], s.argmax(axis=2)[clear])
        # dQ of the first view: the GPU's argmax must attain the max (within the
        # near-tie window), and the gradient through that argmax must match
        i = 0
        j = diff["am"][rows[i]].astype(np.int64)
        assert np.all(s[i, np.arange(N), j] >= s[i].max(axis=1) - 1e-4)
        c = G[b] / nv
        vsel = Vn[np.arange(N) * nv + j]
        ssel = s[i, np.arange(N), j]
        nu = np.linalg.norm(U[i])
        dU = ((c[:, None] * vsel).sum(0) - (c * ssel).sum() * Un[i]) / nu
        dq = dU @ W.astype(np.float64)
        assert np.allclose(diff["dQ"][rows[i]], dq, rtol=1e-4, atol=1e-5 * np.abs(dq).max())


def test_differentiation_sampled_database_views(diff):
    """dP of every view of two database shapes: each view r collects, over all
    query views i whose argmax in its shape is r, c (u_i/|u_i| - s v_r/|v_r|) / |v_r|
    (c = dL/dS / |V(x_b)|), mapped back through W."""
    Q, P, W, G, nv, N = diff["Q"], diff["P"], diff["W"], diff["G"], diff["nv"], diff["N"]
    W64 = W.astype(np.float64)
    U = Q.astype(np.float64) @ W64.T
    Un = U / np.linalg.norm(U, axis=1, keepdims=True)
    b_of = np.arange(Q.shape[0]) // nv
    for p in DIFF_SAMPLED_SHAPES:
        V = P[p].astype(np.float64) @ W64.T
        nvr = np.linalg.norm(V, axis=1)
        Vn = V / nvr[:, None]
        s = Un @ Vn.T                     # [all query views, nv]
        j = diff["am"][:, p].astype(np.int64)
        top2 = np.sort(s, axis=1)[:, -2:]
        assert np.all(s[np.arange(len(j)), j] >= top2[:, 1] - 1e-4)
        c = G[b_of, p] / nv
        dV = np.zeros_like(V)
        for r in range(nv):
            sel = j == r
            if sel.any():
                dV[r] = ((c[sel, None] * Un[sel]).sum(0) - (c[sel] * s[sel, r]).sum() * Vn[r]) / nvr[r]
        dp = dV @ W64
        assert np.allclose(diff["dP"][p], dp, rtol=1e-4, atol=1e-5 * np.abs(dp).max())
