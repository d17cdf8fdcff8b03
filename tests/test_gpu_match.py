"""Differentiable matching (Eq. 3 after a linear view projection) vs the FP64 oracle."""
import numpy as np
import pytest

from oracle import gift_oracle as O

pytestmark = pytest.mark.gpu


def _tie_free(seed, B, Np, nv, din, dout, margin=1e-3, vq=None, counts=None):
    g = np.random.default_rng(seed)
    while True:
        if counts is None:
            counts = np.full(B, nv) if vq is None else g.choice(vq, size=B)
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
        Q = g.standard_normal((off[-1], din)).astype(np.float32)
        P = g.standard_normal((Np, nv, din)).astype(np.float32)
        W = (g.standard_normal((dout, din)) / np.sqrt(din)).astype(np.float32)
        U = Q.astype(np.float64) @ W.T.astype(np.float64)
        V = P.reshape(-1, din).astype(np.float64) @ W.T.astype(np.float64)
        s = O.cosine(U, V).reshape(off[-1], Np, nv)
        top2 = np.sort(s, axis=2)[:, :, -2:]
        if np.min(top2[:, :, 1] - top2[:, :, 0]) > margin:
            G = g.standard_normal((B, Np)).astype(np.float32)
            return Q, off, P, W, G


@pytest.mark.parametrize("with_w", [True, False])
def test_forward_and_argmax(gpu_lib, with_w):
    import torch
    Q, off, P, W, G = _tie_free(1, B=5, Np=37, nv=9, din=48, dout=32 if with_w else 48, margin=1e-4,
                                vq=(3, 9, 14))
    Wt = torch.from_numpy(W).cuda() if with_w else None
    S, am = gpu_lib.match_forward(torch.from_numpy(Q).cuda(), off, torch.from_numpy(P).cuda(), Wt)
    Sr, jr = O.match_forward(Q, off, P, W if with_w else None)
    assert np.allclose(S.cpu().numpy(), Sr, rtol=1e-5, atol=1e-6)
    assert np.array_equal(am.cpu().numpy().astype(np.int64), jr)


@pytest.mark.parametrize("with_w", [True, False])
def test_backward_matches_oracle(gpu_lib, with_w):
    import torch
    Q, off, P, W, G = _tie_free(2, B=4, Np=21, nv=8, din=32, dout=16 if with_w else 32)
    Wd = torch.from_numpy(W).cuda() if with_w else None
    qd, pd = torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda()
    S, am = gpu_lib.match_forward(qd, off, pd, Wd)
    dW, dQ, dP = gpu_lib.match_backward(qd, off, pd, Wd, torch.from_numpy(G).cuda(), am)
    rW, rQ, rP = O.match_backward(Q, off, P, W if with_w else None, G)
    scale = max(np.abs(rQ).max(), np.abs(rP).max())
    assert np.allclose(dQ.cpu().numpy(), rQ, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dP.cpu().numpy(), rP, rtol=1e-4, atol=1e-5 * scale)
    if with_w:
        assert np.allclose(dW.cpu().numpy(), rW, rtol=1e-4, atol=1e-5 * np.abs(rW).max())


@pytest.mark.parametrize("nv,dout,Np", [(70, 16, 6), (5, 144, 6), (1030, 16, 3), (17, 48, 23), (16, 16, 9),
                                         (15, 32, 9)])
def test_backward_ragged_widths(gpu_lib, nv, dout, Np):
    """Gradients with database shapes of 70 and 1,030 views (two and 17 staged 64-view pieces per
    shape on the query side; the 1,030-view shapes take the staged database-side gather instead of
    the per-shape grouping), of 5 views (eight whole shapes per staged step), of 15 to 17 views, and
    projected widths that leave a partial last 128-column slice (16, 48, 144), with the query-side
    step range split into several parts."""
    import torch
    Q, off, P, W, G = _tie_free(8, B=3, Np=Np, nv=nv, din=32, dout=dout, margin=1e-6, counts=(7, 12, 3))
    qd, pd, Wd = torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(), torch.from_numpy(W).cuda()
    S, am = gpu_lib.match_forward(qd, off, pd, Wd)
    dW, dQ, dP = gpu_lib.match_backward(qd, off, pd, Wd, torch.from_numpy(G).cuda(), am)
    rW, rQ, rP = O.match_backward(Q, off, P, W, G)
    scale = max(np.abs(rQ).max(), np.abs(rP).max())
    assert np.allclose(dQ.cpu().numpy(), rQ, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dP.cpu().numpy(), rP, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dW.cpu().numpy(), rW, rtol=1e-4, atol=1e-5 * np.abs(rW).max())


def test_autograd_function(gpu_lib):
    import torch
    Q, off, P, W, G = _tie_free(3, B=3, Np=11, nv=8, din=32, dout=16)
    q = torch.from_numpy(Q).cuda().requires_grad_(True)
    p = torch.from_numpy(P).cuda().requires_grad_(True)
    w = torch.from_numpy(W).cuda().requires_grad_(True)
    S = gpu_lib.GiftMatch.apply(q, off, p, w)
    (S * torch.from_numpy(G).cuda()).sum().backward()
    rW, rQ, rP = O.match_backward(Q, off, P, W, G)
    assert np.allclose(q.grad.cpu().numpy(), rQ, rtol=1e-4, atol=1e-5)
    assert np.allclose(p.grad.cpu().numpy(), rP, rtol=1e-4, atol=1e-5)
    assert np.allclose(w.grad.cpu().numpy(), rW, rtol=1e-4, atol=1e-5 * np.abs(rW).max())


def test_scale_invariants_on_gpu(gpu_lib):
    """<q_i, dS/dq_i> = 0 and <W, dS/dW> = 0 (cosine scale invariance)."""
    import torch
    Q, off, P, W, G = _tie_free(4, B=3, Np=16, nv=8, din=32, dout=16)
    qd, pd, Wd = torch.from_numpy(Q).cuda(), torch.from_numpy(P).cuda(), torch.from_numpy(W).cuda()
    S, am = gpu_lib.match_forward(qd, off, pd, Wd)
    dW, dQ, dP = gpu_lib.match_backward(qd, off, pd, Wd, torch.from_numpy(G).cuda(), am)
    dq = dQ.double().cpu().numpy()
    assert np.abs((Q * dq).sum(1)).max() < 1e-4 * np.abs(dq).max() * np.abs(Q).max() * Q.shape[1] ** 0.5
    assert abs((W * dW.double().cpu().numpy()).sum()) < 1e-4 * np.abs(dW.cpu().numpy()).sum() * np.abs(W).max()


def test_bf16_inputs_forward_backward(gpu_lib):
    """BF16 features and projection (the C4 dtype): compared with the oracle on the
    float64 values of the same BF16 numbers."""
    import torch
    Q, off, P, W, G = _tie_free(5, B=3, Np=19, nv=8, din=64, dout=32, margin=2e-3)
    qb = torch.from_numpy(Q).to(torch.bfloat16).cuda()
    pb = torch.from_numpy(P).to(torch.bfloat16).cuda()
    wb = torch.from_numpy(W).to(torch.bfloat16).cuda()
    Qf, Pf, Wf = (t.float().cpu().numpy() for t in (qb, pb, wb))
    S, am = gpu_lib.match_forward(qb, off, pb, wb)
    Sr, jr = O.match_forward(Qf, off, Pf, Wf)
    assert np.allclose(S.cpu().numpy(), Sr, rtol=1e-5, atol=1e-6)
    assert np.array_equal(am.cpu().numpy().astype(np.int64), jr)
    dW, dQ, dP = gpu_lib.match_backward(qb, off, pb, wb, torch.from_numpy(G).cuda(), am)
    rW, rQ, rP = O.match_backward(Qf, off, Pf, Wf, G)
    scale = max(np.abs(rQ).max(), np.abs(rP).max())
    assert np.allclose(dQ.cpu().numpy(), rQ, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dP.cpu().numpy(), rP, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dW.cpu().numpy(), rW, rtol=1e-4, atol=1e-5 * np.abs(rW).max())
    # autograd returns gradients in the input dtype
    q = qb.clone().requires_grad_(True)
    S2 = gpu_lib.GiftMatch.apply(q, off, pb, wb)
    (S2 * torch.from_numpy(G).cuda()).sum().backward()
    assert q.grad.dtype == torch.bfloat16


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_wide_shapes_several_tiles(gpu_lib, dtype):
    """64 views per database shape and ragged query view counts: the forward's
    short-reduction epilogue (two whole shapes per 128-column tile), the
    query-side gradient GEMM with the A tile generated by four warps (one shape
    per k-block), the database-side segmented sum, BF16 inputs read in place,
    several row tiles with ragged tails — all against the oracle in full."""
    import torch
    Q, off, P, W, G = _tie_free(6, B=4, Np=5, nv=64, din=96, dout=128, margin=1e-5, counts=(40, 100, 64, 57))
    if dtype == "bf16":
        qd, pd, wd = (torch.from_numpy(a).to(torch.bfloat16).cuda() for a in (Q, P, W))
        Q, P, W = (t.float().cpu().numpy() for t in (qd, pd, wd))
    else:
        qd, pd, wd = (torch.from_numpy(a).cuda() for a in (Q, P, W))
    assert off[-1] > 128 and P.shape[0] * P.shape[1] > 256
    S, am = gpu_lib.match_forward(qd, off, pd, wd)
    Sr, jr = O.match_forward(Q, off, P, W)
    assert np.allclose(S.cpu().numpy(), Sr, rtol=1e-5, atol=1e-6)
    assert np.array_equal(am.cpu().numpy().astype(np.int64), jr)
    dW, dQ, dP = gpu_lib.match_backward(qd, off, pd, wd, torch.from_numpy(G).cuda(), am)
    rW, rQ, rP = O.match_backward(Q, off, P, W, G)
    scale = max(np.abs(rQ).max(), np.abs(rP).max())
    assert np.allclose(dQ.cpu().numpy(), rQ, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dP.cpu().numpy(), rP, rtol=1e-4, atol=1e-5 * scale)
    assert np.allclose(dW.cpu().numpy(), rW, rtol=1e-4, atol=1e-5 * np.abs(rW).max())
