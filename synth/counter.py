"""Counter-based view generator, bit-identical in numpy (host) and torch (device).

The 200,000-shape database (52 G feature values) is too large to draw with a
sequential generator on the host once per build pass, so it has a second
recipe whose every value is a pure function of (seed, index): splitmix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to a counter, then integer-only arithmetic up to one
IEEE-exact division. numpy on the host and torch on any device therefore
produce the same bits, and any shape range can be drawn alone.

Recipe (same statistics as the sequential recipe, on a 2^-16 grid):

* h(key, i) = splitmix64 output for state key + (i + 1) * 0x9E3779B97F4A7C15;
  its four 16-bit fields a, b, c, d give e = a + b + c + d - 131070, an
  Irwin-Hall(4) draw with mean 0 and standard deviation 65536 / sqrt(3);
* class centre mu_c[d] = (e * 443) >> 8 with i = c * D + d under the centre
  key (443 / 256 ~ sqrt(3): mu ~ N(0, 1) in units of 2^-16);
* view v of shape s (class s mod C): n[d] = (e * 133) >> 8 with
  i = (s * N_v + v) * D + d under the shape key (133 / 256 ~ 0.3 * sqrt(3):
  noise 0.3), g[d] = max(0, mu_c[d] + n[d]) -- non-negative like ReLU
  activations;
* L2 normalisation: the squared norm sum_d g[d]^2 is an exact int64
  (< 2^50), and x[d] = float32(g[d] / sqrt(norm2)) in float64, where sqrt,
  the division and the rounding to float32 are correctly rounded on both
  sides.

``>>`` is an arithmetic shift (floor division by 256) in numpy and torch.
Nothing here computes a matching score, a quantisation, a ranking or a
re-ranking.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MU_NUM, _NOISE_NUM = 443, 133


def _signed(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


# ------------------------------------------------------------------ numpy
def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def key_of(seed: int) -> int:
    """Generator key of a seed (splitmix64 of seed + 1 steps)."""
    z = np.array([(int(seed) + 1) * _GOLDEN % (1 << 64)], np.uint64)
    return int(_mix_np(z)[0])


def _irwin_hall_np(key: int, idx: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(_GOLDEN)
        h = _mix_np(z)
    m = np.uint64(0xFFFF)
    e = (h & m).astype(np.int64) + ((h >> np.uint64(16)) & m).astype(np.int64) \
        + ((h >> np.uint64(32)) & m).astype(np.int64) + (h >> np.uint64(48)).astype(np.int64)
    return e - 131070


def centres_np(n_classes: int, dim: int, centre_seed: int) -> np.ndarray:
    """Class centres on the 2^-16 grid, int64 [C, D]."""
    idx = np.arange(n_classes * dim, dtype=np.int64)
    return ((_irwin_hall_np(key_of(centre_seed), idx) * _MU_NUM) >> 8).reshape(n_classes, dim)


def _views_np(first: int, n: int, nv: int, dim: int, mu: np.ndarray, key: int) -> np.ndarray:
    C = mu.shape[0]
    out = np.empty((n, nv, dim), np.float32)
    d = np.arange(dim, dtype=np.int64)
    for j in range(n):
        s = first + j
        idx = (np.int64(s) * nv + np.arange(nv, dtype=np.int64))[:, None] * dim + d[None, :]
        g = np.maximum(mu[s % C][None, :] + ((_irwin_hall_np(key, idx) * _NOISE_NUM) >> 8), 0)
        n2 = (g * g).sum(axis=1, keepdims=True)
        n2[n2 == 0] = 1
        out[j] = (g.astype(np.float64) / np.sqrt(n2.astype(np.float64))).astype(np.float32)
    return out


def shape_views_np(first: int, n: int, nv: int, dim: int, n_classes: int, seed: int, centre_seed: int,
                   threads: int | None = None) -> np.ndarray:
    """Views of shapes [first, first + n): float32 [n, nv, dim] (host, threaded)."""
    mu = centres_np(n_classes, dim, centre_seed)
    key = key_of(seed)
    threads = threads or min(32, os.cpu_count() or 1)
    step = max(1, min(64, (n + threads - 1) // threads))
    spans = [(f, min(step, first + n - f)) for f in range(first, first + n, step)]
    if len(spans) == 1 or threads == 1:
        return np.concatenate([_views_np(f, m, nv, dim, mu, key) for f, m in spans]) if spans else \
            np.empty((0, nv, dim), np.float32)
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda sp: _views_np(sp[0], sp[1], nv, dim, mu, key), spans))
    return np.concatenate(parts)


# ------------------------------------------------------------------ torch
def _lsr(z, s: int):
    """Logical right shift of int64 bit patterns."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix_t(z):
    z = (z ^ _lsr(z, 30)) * _signed(_M1)
    z = (z ^ _lsr(z, 27)) * _signed(_M2)
    return z ^ _lsr(z, 31)


def _irwin_hall_t(key: int, idx):
    h = _mix_t(idx * _signed(_GOLDEN) + _signed((key + _GOLDEN) % (1 << 64)))
    m = 0xFFFF
    return (h & m) + (_lsr(h, 16) & m) + (_lsr(h, 32) & m) + _lsr(h, 48) - 131070


def centres_torch(n_classes: int, dim: int, centre_seed: int, device):
    import torch
    idx = torch.arange(n_classes * dim, dtype=torch.int64, device=device)
    return ((_irwin_hall_t(key_of(centre_seed), idx) * _MU_NUM) >> 8).view(n_classes, dim)


def shape_views_torch(first: int, n: int, nv: int, dim: int, n_classes: int, seed: int, centre_seed: int,
                      device="cuda", mu=None, out=None):
    """The same views as shape_views_np, drawn on a torch device: float32 [n, nv, dim].

    Works in pieces of up to 64 shapes (about 2 GB of int64 temporaries).
    """
    import torch
    if mu is None:
        mu = centres_torch(n_classes, dim, centre_seed, device)
    key = key_of(seed)
    if out is None:
        out = torch.empty((n, nv, dim), dtype=torch.float32, device=device)
    cls_all = torch.arange(first, first + n, device=device, dtype=torch.int64) % n_classes
    d = torch.arange(dim, dtype=torch.int64, device=device)
    v = torch.arange(nv, dtype=torch.int64, device=device)
    for j0 in range(0, n, 64):
        m = min(64, n - j0)
        s = torch.arange(first + j0, first + j0 + m, dtype=torch.int64, device=device)
        idx = ((s[:, None] * nv + v[None, :])[:, :, None] * dim + d[None, None, :])
        g = mu[cls_all[j0:j0 + m]][:, None, :] + ((_irwin_hall_t(key, idx) * _NOISE_NUM) >> 8)
        g = torch.clamp_min(g, 0)
        n2 = (g * g).sum(dim=2, keepdim=True)
        n2 = torch.where(n2 == 0, torch.ones_like(n2), n2)
        out[j0:j0 + m] = (g.to(torch.float64) / torch.sqrt(n2.to(torch.float64))).to(torch.float32)
    return out
