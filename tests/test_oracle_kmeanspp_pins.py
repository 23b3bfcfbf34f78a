"""Pins of the oracle's K-means++ seeding (the initial seeds Section 4.2
takes from Arthur & Vassilvitskii 2007): the independent numpy recipe in
inputs.kmeanspp, hand-worked draws on a line, the D^2 sampling distribution
over a grid of uniforms, the distance to the closest seed (not the last
one), and the all-duplicates case."""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs


@pytest.mark.parametrize("case", ["blobs", "mixture", "mnist_like", "manifolds"])
def test_equals_numpy_recipe(case):
    if case == "blobs":
        X, _ = inputs.blobs(N=3000, D=16, n_blobs=7, seed=2)
        L, seed = 20, 2
    elif case == "mixture":
        X, _ = inputs.mixture(4000, 9, 30, seed=5)
        L, seed = 30, 5
    elif case == "mnist_like":
        X, _ = inputs.mnist_like(N=2500)
        L, seed = 10, 1810
    else:
        X, _ = inputs.manifolds(N=5000, D=32, n_clusters=20)
        L, seed = 50, 1810
    first, u = inputs.kmeanspp_draws(X.shape[0], L, seed)
    np.testing.assert_array_equal(oracle.kmeanspp(X, L, first, u), inputs.kmeanspp(X, L, seed=seed))


def test_hand_worked_draws_on_a_line():
    # points 0, 1, 3 on a line, first seed 0: D^2 = (0, 1, 9), total 10; the
    # running sums 0, 1, 10 are first above r = 10 u at p = 1 for u < 0.1
    # (u = 0 included: a point at distance 0 is never drawn) and at p = 2 above
    X = np.array([[0.0], [1.0], [3.0]], np.float32)
    for u, want in [(0.0, 1), (0.05, 1), (0.0999, 1), (0.1, 2), (0.5, 2), (0.999, 2)]:
        assert oracle.kmeanspp(X, 2, 0, [u])[1] == want
    # points 0, 1, 3, 3: D^2 = (0, 1, 9, 9), running sums 0, 1, 10, 19, so
    # u = 0.95 (r = 18.05) draws point 3; the next draw measures distances to
    # the closest of both seeds, D^2 = (0, 1, 0, 0), and only point 1 remains
    X4 = np.array([[0.0], [1.0], [3.0], [3.0]], np.float32)
    assert list(oracle.kmeanspp(X4, 3, 0, [0.95, 0.0])) == [0, 3, 1]
    assert list(oracle.kmeanspp(X4, 3, 0, [0.95, 0.999])) == [0, 3, 1]


def test_draw_frequencies_follow_d_squared():
    """Over uniforms on a fine grid, point p is drawn for a share of the grid
    equal to D(x_p)^2 / sum D^2 (to within one grid step)."""
    g = inputs.rng(4)
    X = g.normal(size=(12, 3)).astype(np.float32)
    M = 4000
    counts = np.zeros(12)
    for j in range(M):
        counts[oracle.kmeanspp(X, 2, 5, [(j + 0.5) / M])[1]] += 1
    d2 = ((X.astype(np.float64) - X[5].astype(np.float64)) ** 2).sum(1)
    np.testing.assert_allclose(counts / M, d2 / d2.sum(), atol=1.5 / M)
    assert counts[5] == 0


def test_all_points_identical():
    X = np.ones((10, 4), np.float32)
    s = oracle.kmeanspp(X, 4, 3, [0.0, 0.55, 0.999])
    assert list(s) == [3, 0, 5, 9]


def test_rejects_bad_arguments():
    X = np.zeros((5, 2), np.float32)
    with pytest.raises(ValueError):
        oracle.kmeanspp(X, 6, 0, np.zeros(5))
    with pytest.raises(ValueError):
        oracle.kmeanspp(X, 2, 7, [0.5])
