"""Seeded synthetic triangle meshes for the projection front end.

Each mesh is a closed, star-shaped surface: a latitude/longitude grid whose
radius is 1 + a seeded sum of a few smooth angular bumps, then stretched,
rotated about z and shifted by seeded amounts (so that the scale and
translation normalisation of the renderer has work to do). Class c shares its
bump pattern; shapes of a class differ by small seeded perturbations.

Nothing here renders or normalises: the meshes are inputs.
"""
from __future__ import annotations

import numpy as np


def _gen(seed: int, block: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(block)])


def star_mesh(shape_id: int, n_classes: int, seed: int, n_lat: int = 24, n_lon: int = 48):
    """One mesh: (vertices float32 [V, 3], triangles int32 [T, 3]), V = (n_lat - 1) * n_lon + 2."""
    cls = shape_id % n_classes
    gc = _gen(seed, 100000 + cls)
    gs = _gen(seed, shape_id)
    nb = 5
    amp = gc.uniform(0.05, 0.35, nb) * (1.0 + 0.1 * gs.standard_normal(nb))
    fa = gc.integers(1, 5, nb)
    fb = gc.integers(1, 4, nb)
    ph = gc.uniform(0, 2 * np.pi, (nb, 2)) + 0.1 * gs.standard_normal((nb, 2))
    theta = np.pi * np.arange(1, n_lat) / n_lat            # polar angle, poles excluded
    phi = 2 * np.pi * np.arange(n_lon) / n_lon
    T, P = np.meshgrid(theta, phi, indexing="ij")
    r = np.ones_like(T)
    for k in range(nb):
        r += amp[k] * np.cos(fa[k] * P + ph[k, 0]) * np.sin(fb[k] * T + ph[k, 1])
    r = np.maximum(r, 0.2)
    ring = np.stack([r * np.sin(T) * np.cos(P), r * np.sin(T) * np.sin(P), r * np.cos(T)], axis=-1).reshape(-1, 3)
    north = np.array([[0.0, 0.0, 1.0]])
    south = np.array([[0.0, 0.0, -1.0]])
    V = np.concatenate([north, ring, south])
    stretch = gs.uniform(0.6, 1.6, 3)
    ang = gs.uniform(0, 2 * np.pi)
    Rz = np.array([[np.cos(ang), -np.sin(ang), 0], [np.sin(ang), np.cos(ang), 0], [0, 0, 1]])
    V = (V * stretch) @ Rz.T * gs.uniform(0.5, 4.0) + gs.uniform(-3, 3, 3)
    tris = []
    idx = lambda i, j: 1 + i * n_lon + (j % n_lon)  # ring vertex (latitude row i, longitude j)
    for j in range(n_lon):
        tris.append((0, idx(0, j), idx(0, j + 1)))
        tris.append((len(V) - 1, idx(n_lat - 2, j + 1), idx(n_lat - 2, j)))
    for i in range(n_lat - 2):
        for j in range(n_lon):
            a, b, c, d = idx(i, j), idx(i, j + 1), idx(i + 1, j), idx(i + 1, j + 1)
            tris.append((a, c, b))
            tris.append((b, c, d))
    return V.astype(np.float32), np.asarray(tris, np.int32)


def mesh_batch(first: int, n: int, n_classes: int, seed: int, n_lat: int = 24, n_lon: int = 48):
    """Meshes [first, first + n) packed: (vertices [sum V, 3], triangles [sum T, 3] local to
    their mesh, vertex offsets int64 [n + 1], triangle offsets int64 [n + 1])."""
    vs, ts = [], []
    for s in range(first, first + n):
        v, t = star_mesh(s, n_classes, seed, n_lat, n_lon)
        vs.append(v)
        ts.append(t)
    voff = np.concatenate([[0], np.cumsum([len(v) for v in vs])]).astype(np.int64)
    toff = np.concatenate([[0], np.cumsum([len(t) for t in ts])]).astype(np.int64)
    return np.concatenate(vs), np.concatenate(ts), voff, toff
