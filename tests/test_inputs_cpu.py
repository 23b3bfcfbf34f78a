"""The seeded input recipes: shapes, determinism, and the structure each
generator promises (equal or Zipf cluster sizes, the [0, 1] feature range of
the MNIST-shaped data, the 16-dimensional affine span of a curved 8-dim
manifold cluster, the largest-cluster share of a mixture, valid graphs and
simplex rows, K-means++ seeds that are point indices)."""
import numpy as np
import pytest

from paper_1810_13044_gb300 import inputs


@pytest.mark.parametrize("N,w", [(10, [1, 1, 1]), (2000, [1] * 5), (1000, [0.7, 0.2, 0.05, 0.05]),
                                 (7, [100, 1, 1, 1, 1, 1, 1]), (12345, np.arange(1, 101) ** -1.1)])
def test_split_sizes(N, w):
    s = inputs._split_sizes(N, np.asarray(w, dtype=np.float64))
    assert s.sum() == N and s.min() >= 1 and len(s) == len(w)
    raw = np.asarray(w, dtype=np.float64) / np.sum(w) * N
    if raw.min() >= 1.0:   # no cluster was lifted to its minimum of one point
        assert np.all(np.abs(s - raw) < 1.0)


def test_blobs_shape_sizes_and_seed():
    X, y = inputs.blobs()
    assert X.shape == (2000, 16) and X.dtype == np.float32 and X.flags["C_CONTIGUOUS"]
    assert np.array_equal(np.bincount(y), [400] * 5)
    X2, y2 = inputs.blobs()
    assert np.array_equal(X, X2) and np.array_equal(y, y2)
    X3, _ = inputs.blobs(seed=7)
    assert not np.array_equal(X, X3)
    # unit variance around each centre (400 draws per feature: standard error ~0.07)
    for b in range(5):
        v = X[y == b].astype(np.float64).var(axis=0, ddof=1)
        assert 0.85 < v.mean() < 1.15


def test_mnist_like_range_and_clusters():
    X, y = inputs.mnist_like(N=3000)
    assert X.shape == (3000, 784) and X.dtype == np.float32
    assert np.array_equal(np.bincount(y), [300] * 10)
    assert X.min() == 0.0 and X.max() == 1.0
    lo, hi = X.min(axis=0), X.max(axis=0)
    varying = hi > lo
    assert varying.mean() > 0.99
    assert np.all(lo[varying] == 0.0) and np.all(hi[varying] == 1.0)


def test_manifolds_zipf_sizes_and_affine_span():
    N, D, C = 20000, 128, 100
    X, y = inputs.manifolds(N=N, D=D, n_clusters=C)
    assert X.shape == (N, D) and X.dtype == np.float32
    sizes = np.bincount(y, minlength=C)
    assert sizes.sum() == N and sizes.min() >= 1
    expect = np.arange(1, C + 1) ** -1.1
    expect = expect / expect.sum() * N
    assert np.all(np.abs(sizes - expect) <= 1.0)
    assert 0.22 < sizes[0] / N < 0.24          # the largest cluster holds about 23 %
    # x = c + U t + 0.3 V (t*t) lies in the affine span of the 16 columns of [U V]
    P = X[y == 0].astype(np.float64)
    sv = np.linalg.svd(P - P.mean(axis=0), compute_uv=False)
    assert sv[15] > 1e3 * sv[16]


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_mixture_largest_share(seed):
    N = 5000
    X, y = inputs.mixture(N, 16, 6, seed)
    share = np.bincount(y).max() / N
    assert 0.6 - 1.0 / N <= share <= 0.8 + 1.0 / N
    assert X.shape == (N, 16) and X.dtype == np.float32


def test_kmeanspp_indices():
    X, _ = inputs.blobs()
    m = inputs.kmeanspp(X, 5)
    assert m.dtype == np.int32 and m.shape == (5,)
    assert len(set(m.tolist())) == 5 and m.min() >= 0 and m.max() < X.shape[0]
    assert np.array_equal(m, inputs.kmeanspp(X, 5))
    with pytest.raises(ValueError):
        inputs.kmeanspp(X, 0)


@pytest.mark.parametrize("N,k", [(2, 1), (5, 4), (300, 7), (70000, 5)])
def test_random_graph_is_knn_shaped(N, k):
    row_ptr, col, w = inputs.random_graph(N, k, seed=11, weighted=True)
    assert np.array_equal(row_ptr, np.arange(N + 1) * k)
    C = col.reshape(N, k).astype(np.int64)
    assert C.min() >= 0 and C.max() < N
    assert not np.any(C == np.arange(N)[:, None])
    Cs = np.sort(C, axis=1)
    assert np.all(Cs[:, 1:] != Cs[:, :-1])
    assert w.shape == (N * k,) and w.min() >= 0.05 and w.max() <= 1.0


def test_simplex_rows_and_unary():
    Z = inputs.random_simplex_rows(1000, 7, seed=2)
    assert Z.dtype == np.float32 and Z.min() >= 0.0
    assert np.abs(Z.astype(np.float64).sum(axis=1) - 1.0).max() < 1e-6
    A = inputs.random_unary(1000, 7, seed=2)
    assert A.dtype == np.float32 and A.min() > 0.0 and A.max() <= 1.0
