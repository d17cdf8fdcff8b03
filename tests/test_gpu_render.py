"""Projection front end (Sec. 2.1) on the GPU against the float64 oracle renderer.

Pixels whose centre lies within a hair of a triangle edge (relative edge function
below 1e-5 in the oracle) or where two surfaces are within 1e-5 in depth may
resolve either way in FP32; everywhere else coverage is identical and depths
agree within 1e-4 (FP32 screen coordinates carry ~1e-7 of position error, which
the depth gradient of a surface seen at a grazing angle multiplies; depth images
are quantised far more coarsely before feature extraction).
"""
import numpy as np
import pytest

from oracle import gift_oracle as O
from synth.meshes import mesh_batch

pytestmark = pytest.mark.gpu


def _unstable(V, T, n_az, n_el, H, W, eps=1e-5):
    """Oracle-side mask [N_v, H, W] of pixels near an edge or a depth tie."""
    c, s = O.normalize_mesh(V, T)
    P = (np.asarray(V, np.float64) - c) * s
    _, f, r, u = O.view_frames(n_az, n_el)
    xs = -1 + (2 * np.arange(W) + 1) / W
    ys = 1 - (2 * np.arange(H) + 1) / H
    X, Y = np.meshgrid(xs, ys)
    out = np.zeros((len(f), H, W), bool)
    for v in range(len(f)):
        S = np.stack([P @ r[v], P @ u[v], P @ f[v] + 1.0], axis=1)
        best = np.full((H, W), 2.0)
        second = np.full((H, W), 2.0)
        for t in np.asarray(T):
            a, b, cc = S[t[0]], S[t[1]], S[t[2]]
            area = (b[0] - a[0]) * (cc[1] - a[1]) - (b[1] - a[1]) * (cc[0] - a[0])
            if area == 0:
                continue
            if area < 0:
                b, cc, area = cc, b, -area
            ea = ((cc[0] - b[0]) * (Y - b[1]) - (cc[1] - b[1]) * (X - b[0])) / area
            eb = ((a[0] - cc[0]) * (Y - cc[1]) - (a[1] - cc[1]) * (X - cc[0])) / area
            ec = ((b[0] - a[0]) * (Y - a[1]) - (b[1] - a[1]) * (X - a[0])) / area
            m = np.minimum(np.minimum(ea, eb), ec)
            out[v] |= np.abs(m) < eps
            z = np.where(m >= 0, ea * a[2] + eb * b[2] + ec * cc[2], 2.0)
            second = np.where(z < best, best, np.minimum(second, z))
            best = np.minimum(best, z)
        out[v] |= (best < 2.0) & ((second - best) < eps)  # two surfaces within eps in depth
    return out


@pytest.mark.parametrize("n_az,n_el,H,W", [(4, 2, 24, 20), (8, 8, 16, 16)])
def test_depth_views_match_oracle(gpu_lib, n_az, n_el, H, W):
    V, T, vo, to = mesh_batch(0, 3, 5, 21, n_lat=8, n_lon=12)
    out = gpu_lib.render_views(V, T, vo, to, n_az, n_el, H, W).cpu().numpy()
    assert out.shape == (3, n_az * n_el, H, W)
    for m in range(3):
        Vm, Tm = V[vo[m]:vo[m + 1]], T[to[m]:to[m + 1]]
        ref = O.render_depth(Vm, Tm, n_az, n_el, H, W)
        bad = _unstable(Vm, Tm, n_az, n_el, H, W)
        ok = ~bad
        assert ok.mean() > 0.9
        assert np.array_equal(out[m][ok] < 2, ref[ok] < 2)
        err = np.abs(out[m][ok] - ref[ok])
        assert err.max() < 1e-4 and np.median(err) < 1e-6


def test_device_inputs_and_invariance(gpu_lib):
    import torch
    V, T, vo, to = mesh_batch(3, 2, 5, 22, n_lat=10, n_lon=16)
    a = gpu_lib.render_views(torch.from_numpy(V).cuda(), torch.from_numpy(T).cuda(), vo, to, 4, 4, 32, 32)
    V2 = V.copy()
    V2[vo[1]:vo[2]] = V2[vo[1]:vo[2]] * 2.5 + np.array([1.0, -4.0, 0.5], np.float32)  # move and scale mesh 1
    b = gpu_lib.render_views(V2, T, vo, to, 4, 4, 32, 32)
    assert torch.equal(a[0], b[0])
    assert (a[1] - b[1]).abs().max().item() < 1e-4


def test_bad_triangle_rejected(gpu_lib):
    V, T, vo, to = mesh_batch(0, 2, 5, 23, n_lat=6, n_lon=8)
    T = T.copy()
    T[to[1] + 2, 1] = vo[2] - vo[1]  # one past the second mesh's vertices
    with pytest.raises(gpu_lib.GiftError):
        gpu_lib.render_views(V, T, vo, to, 2, 2, 8, 8)
