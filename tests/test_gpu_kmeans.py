"""GPU Lloyd k-means (the off-line vocabulary) against the float64 oracle."""
import numpy as np
import pytest

from oracle import gift_oracle as O
from synth import shape_views, kmeans_init_rows

pytestmark = pytest.mark.gpu


def _data():
    return shape_views(0, 64, 16, 64, 5, 1501, 4501).reshape(-1, 64)  # 1,024 rows, 5 classes


def test_kmeans_matches_oracle(gpu_lib):
    import torch
    X = _data()
    init = kmeans_init_rows(len(X), 32, 7)
    C = gpu_lib.kmeans(torch.from_numpy(X).cuda(), init, iters=6).cpu().numpy()
    ref = O.kmeans_lloyd(X, init, 6)
    assert np.abs(C - ref).max() < 1e-5


def test_kmeans_reseeds_empty_centres_and_takes_host_input(gpu_lib):
    X = _data()
    init = np.array([0, 0, 0, 17, 400, 800], np.int32)  # two duplicate centres start empty
    C = gpu_lib.kmeans(X, init, iters=3).cpu().numpy()
    ref = O.kmeans_lloyd(X, init, 3)
    assert np.abs(C - ref).max() < 1e-5
    assert np.array_equal(gpu_lib.kmeans(X, init, iters=0).cpu().numpy(), X[init])


def test_kmeans_rejects_bad_rows(gpu_lib):
    X = _data()
    with pytest.raises(gpu_lib.GiftError):
        gpu_lib.kmeans(X, np.array([0, len(X)], np.int32), iters=1)
