"""Seeded synthetic inputs for the SLK hot path.

This module only draws random numbers and lays them out; it holds none of the
clustering method's arithmetic.  Both the CUDA path and the FP64 oracle are fed
from here, so that they see bit-identical inputs.

Workloads (stand-ins for the paper's datasets of Table 1, which are not
available here; shapes follow Table 1 and the experiments of Section 4):

* ``blobs``      -- N=2000, D=16, 5 isotropic unit-variance Gaussian blobs with
                    centres ~ N(0, 25 I), equal sizes (MNIST-small sized N).
* ``mnist_like`` -- N=70000, D=784 in [0, 1], 10 equal clusters; each is a
                    10-dim latent Gaussian pushed through a fixed random
                    2-layer ReLU map, then every feature is min-max scaled
                    (the shape of MNIST in Table 1).
* ``manifolds``  -- N=1e6, D=128, L=100 clusters on curved 8-dim manifolds
                    with Zipf(1.1) cluster sizes.
* ``mixture``    -- one imbalanced Gaussian mixture instance (largest cluster
                    60-80 %) used by the batched form.

Points are emitted in a seeded random order (as a real dataset would be), and
the generating cluster id of each point is returned for sanity checks only.

The initial modes of Algorithm 1 are K-means++ seeds (Section 4.2 cites
Arthur & Vassilvitskii 2007 for them); :func:`kmeanspp` draws them here, once,
so that every implementation starts from the same point indices.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "blobs", "mnist_like", "manifolds", "mixture", "kmeanspp", "kmeanspp_draws",
    "random_graph", "random_unary", "random_simplex_rows", "WORKLOADS",
]


def rng(seed: int) -> np.random.Generator:
    """The one random source used by every generator (PCG64, seeded)."""
    return np.random.Generator(np.random.PCG64(seed))


def _shuffle(g: np.random.Generator, X: np.ndarray, y: np.ndarray):
    perm = g.permutation(X.shape[0])
    return np.ascontiguousarray(X[perm]), np.ascontiguousarray(y[perm])


def _split_sizes(N: int, weights: np.ndarray) -> np.ndarray:
    """Integer cluster sizes summing to N, proportional to ``weights``
    (largest-remainder rounding, every cluster at least one point)."""
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    raw = w * N
    sizes = np.maximum(np.floor(raw).astype(np.int64), 1)
    rem = N - int(sizes.sum())
    if rem > 0:
        order = np.argsort(-(raw - np.floor(raw)), kind="stable")
        sizes[order[:rem]] += 1
    elif rem < 0:
        order = np.argsort(-sizes, kind="stable")
        i = 0
        while rem < 0:
            j = order[i % len(order)]
            if sizes[j] > 1:
                sizes[j] -= 1
                rem += 1
            i += 1
    return sizes


def blobs(N: int = 2000, D: int = 16, n_blobs: int = 5, centre_var: float = 25.0,
          seed: int = 1810):
    """Isotropic unit-variance Gaussian blobs, centres ~ N(0, centre_var I),
    equal sizes (the last blob takes the remainder)."""
    g = rng(seed)
    centres = g.normal(0.0, np.sqrt(centre_var), size=(n_blobs, D))
    sizes = _split_sizes(N, np.ones(n_blobs))
    y = np.repeat(np.arange(n_blobs, dtype=np.int32), sizes)
    X = centres[y] + g.normal(0.0, 1.0, size=(N, D))
    return _shuffle(g, X.astype(np.float32), y)


def _dyadic(x: np.ndarray, bits: int, lim: float) -> np.ndarray:
    """x clipped to [-lim, lim] and rounded to a multiple of 2^-bits (float64)."""
    return np.round(np.clip(x, -lim, lim) * 2.0 ** bits) / 2.0 ** bits


def mnist_like(N: int = 70000, D: int = 784, n_clusters: int = 10, latent: int = 10,
               hidden: int = 256, seed: int = 1810):
    """Latent Gaussians u ~ N(mu_c, I) with mu_c ~ N(0, 9 I), a fixed random
    map x = W2 ReLU(W1 u + b1) + b2, then per-feature min-max to [0, 1].

    Every random factor is rounded to a short dyadic grid (and clipped far
    out in its tail) so that each product and every partial sum of the two
    matrix products is exact in float64: the result does not depend on the
    order in which a BLAS library adds, so x86 and Arm hosts produce the
    same bits.  Grids and bounds: mu, u - mu, W1, b1, b2 on 2^-16, W2 on
    2^-12, the hidden layer rounded to 2^-20; every sum then stays below
    2^50 units of its grid."""
    g = rng(seed)
    mu = _dyadic(g.normal(0.0, 3.0, size=(n_clusters, latent)), 16, 24.0)
    W1 = _dyadic(g.normal(0.0, np.sqrt(1.0 / latent), size=(hidden, latent)), 16, 2.0)
    b1 = _dyadic(g.normal(0.0, 1.0, size=hidden), 16, 8.0)
    W2 = _dyadic(g.normal(0.0, np.sqrt(1.0 / hidden), size=(D, hidden)), 12, 0.5)
    b2 = _dyadic(g.normal(0.0, 0.1, size=D), 16, 1.0)
    sizes = _split_sizes(N, np.ones(n_clusters))
    y = np.repeat(np.arange(n_clusters, dtype=np.int32), sizes)
    U = mu[y] + _dyadic(g.normal(0.0, 1.0, size=(N, latent)), 16, 8.0)
    H = _dyadic(np.maximum(U @ W1.T + b1, 0.0), 20, 1e6)
    X = H @ W2.T + b2
    lo = X.min(axis=0)
    hi = X.max(axis=0)
    X = (X - lo) / np.where(hi > lo, hi - lo, 1.0)
    return _shuffle(g, X.astype(np.float32), y)


def manifolds(N: int = 1_000_000, D: int = 128, n_clusters: int = 100, intrinsic: int = 8,
              zipf: float = 1.1, spread: float = 3.0, curvature: float = 0.3, seed: int = 1810):
    """Clusters on curved ``intrinsic``-dim manifolds,
    x = c_l + U_l t + curvature * V_l (t*t), t ~ N(0, I), with U_l, V_l random
    orthonormal D x intrinsic frames, c_l ~ N(0, spread^2 I) and cluster sizes
    proportional to l^(-zipf)."""
    g = rng(seed)
    sizes = _split_sizes(N, np.arange(1, n_clusters + 1, dtype=np.float64) ** (-zipf))
    y = np.repeat(np.arange(n_clusters, dtype=np.int32), sizes)
    X = np.empty((N, D), dtype=np.float32)
    start = 0
    for l in range(n_clusters):
        n = int(sizes[l])
        c = g.normal(0.0, spread, size=D)
        U = np.linalg.qr(g.normal(size=(D, intrinsic)))[0]
        V = np.linalg.qr(g.normal(size=(D, intrinsic)))[0]
        t = g.normal(0.0, 1.0, size=(n, intrinsic))
        X[start:start + n] = (c + t @ U.T + curvature * (t * t) @ V.T).astype(np.float32)
        start += n
    return _shuffle(g, X, y)


def mixture(N: int, D: int, n_clusters: int, seed: int, largest=(0.6, 0.8)):
    """Imbalanced Gaussian mixture: one cluster holds a fraction drawn
    uniformly from ``largest`` of the points, the rest share the remainder at
    random; centres ~ N(0, 16 I), unit variance."""
    g = rng(seed)
    frac = g.uniform(*largest)
    rest = g.dirichlet(np.ones(max(n_clusters - 1, 1))) * (1.0 - frac)
    w = np.concatenate([[frac], rest])[:n_clusters]
    sizes = _split_sizes(N, w)
    centres = g.normal(0.0, 4.0, size=(n_clusters, D))
    y = np.repeat(np.arange(n_clusters, dtype=np.int32), sizes)
    X = centres[y] + g.normal(0.0, 1.0, size=(N, D))
    return _shuffle(g, X.astype(np.float32), y)


def kmeanspp_draws(N: int, L: int, seed: int = 1810):
    """The random draws of K-means++ seeding: the first seed's index (uniform
    over the N points) and L - 1 uniforms in [0, 1), one per further seed."""
    g = rng(seed)
    first = int(g.integers(N))
    u = g.random(max(L - 1, 0))
    return first, u


def kmeanspp(X: np.ndarray, L: int, seed: int = 1810, chunk: int = 65536) -> np.ndarray:
    """K-means++ seeding (Arthur & Vassilvitskii 2007): the first seed is a
    uniformly drawn point, each next one is drawn with probability
    proportional to the squared distance to the closest seed so far -- the
    point at which the running sum of those squared distances first exceeds
    u * their total, u the next uniform of :func:`kmeanspp_draws` (when every
    distance is zero: point floor(u N)).  Returns ``L`` point indices (int32)."""
    N = X.shape[0]
    if not 1 <= L <= N:
        raise ValueError("need 1 <= L <= N")
    first, u = kmeanspp_draws(N, L, seed)
    seeds = [first]
    closest = np.full(N, np.inf)
    for i in range(1, L):
        c = X[seeds[-1]].astype(np.float64)
        for s in range(0, N, chunk):
            diff = X[s:s + chunk].astype(np.float64) - c
            np.minimum(closest[s:s + chunk], np.einsum("ij,ij->i", diff, diff),
                       out=closest[s:s + chunk])
        total = closest.sum()
        if total <= 0.0:
            seeds.append(min(int(u[i - 1] * N), N - 1))
            continue
        idx = int(np.searchsorted(np.cumsum(closest), u[i - 1] * total, side="right"))
        seeds.append(min(idx, N - 1))
    return np.array(seeds, dtype=np.int32)


def random_graph(N: int, k: int, seed: int, weighted: bool = False):
    """A random directed graph in CSR form with exactly ``k`` distinct
    neighbours q != p per row (the shape of a kNN graph).  Returns
    ``(row_ptr int64[N+1], col_idx int32[N*k], w float32[N*k] or None)``."""
    g = rng(seed)
    if k > N - 1:
        raise ValueError("k must be <= N-1")
    col = np.empty((N, k), dtype=np.int64)
    m = 4 * k + 8
    for s in range(0, N, 1 << 16):
        n = min(1 << 16, N - s)
        draw = g.integers(0, N - 1, size=(n, m))
        p = np.arange(s, s + n)[:, None]
        draw = draw + (draw >= p)                      # skip the row itself
        # keep the first k distinct values of each row, in draw order
        order = np.argsort(draw, axis=1, kind="stable")
        sv = np.take_along_axis(draw, order, 1)
        first = np.ones_like(sv, dtype=bool)
        first[:, 1:] = sv[:, 1:] != sv[:, :-1]
        key = np.where(first, order, m + 1)
        pos = np.sort(key, axis=1)[:, :k]
        ok = pos[:, -1] <= m
        rows_ok = np.nonzero(ok)[0]
        col[s + rows_ok] = np.take_along_axis(draw[rows_ok], pos[rows_ok], 1)
        for i in np.nonzero(~ok)[0]:                   # tiny N: a permutation
            others = np.setdiff1d(np.arange(N), [s + i])
            col[s + i] = g.permutation(others)[:k]
    row_ptr = (np.arange(N + 1, dtype=np.int64) * k)
    w = g.uniform(0.05, 1.0, size=N * k).astype(np.float32) if weighted else None
    return row_ptr, col.reshape(-1).astype(np.int32), w


def random_unary(N: int, L: int, seed: int) -> np.ndarray:
    """Unary-term-like values in (0, 1] (float32, N x L)."""
    g = rng(seed)
    return g.uniform(1e-3, 1.0, size=(N, L)).astype(np.float32)


def random_simplex_rows(N: int, L: int, seed: int) -> np.ndarray:
    """Rows drawn uniformly on the probability simplex (float32, N x L)."""
    g = rng(seed)
    Z = g.dirichlet(np.ones(L), size=N)
    return Z.astype(np.float32)


# Named workloads: (generator, kwargs, L, k, affinity, precision)
WORKLOADS = {
    "blobs_2000x16_L5": dict(gen="blobs", kw={}, L=5, k=5, affinity="binary", lam=1.0),
    "mnist_like_70000x784_L10": dict(gen="mnist_like", kw={}, L=10, k=5, affinity="binary", lam=1.0),
    "manifolds_1e6x128_L100": dict(gen="manifolds", kw={}, L=100, k=10, affinity="heat", lam=1.0),
}
