"""Whole-solve parity at the scale of the workloads: the CUDA path (through
the C-ABI) against the FP64 oracle on the same seeded points.

* 70000 x 784, L = 10, k = 5, binary affinity (MNIST-shaped): the oracle's
  exact kNN graph of these points is stored in tests/golden (written by
  tests/golden/make_mnist_like_knn.py, which calls only the oracle; the
  SHA-256 of the points it was computed on is checked, and on a mismatch
  the graph is recomputed here by the oracle on all host cores).
* 20000 x 128, L = 100, k = 10, heat affinity, bfloat16 tensor-core
  candidates (the precision workload's generator at N = 20000): the oracle
  computes the exact graph here.

Both sides start from the same K-means++ seeds and the oracle's sigma
(median kNN distance, Section 4.2).  Checks: the GPU's whole kNN graph
equals the oracle's (a different index only between distances equal within
the float32 rounding bound of a D-term sum), the GPU's sigma, then the
solve: the same number of outer iterations, identical mode indices and
labels (a difference only where the oracle's own values are a near-tie, and
counted), Z within 1e-5 max-abs and E within 1e-6 relative.
"""
import hashlib
import os

import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs
from parity_checks import compare_solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN_MNIST = os.path.join(HERE, "golden", "mnist_like_70000x784_k5_knn.npz")


@pytest.fixture(scope="module")
def slk():
    from paper_1810_13044_gb300 import build, slk as _slk
    build.build()
    return _slk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def oracle_graph(X, k, golden=None):
    """The oracle's exact kNN graph (idx, d2) of X; from the stored golden
    when it was computed on these very points."""
    if golden is not None and os.path.exists(golden):
        z = np.load(golden)
        sha = hashlib.sha256(np.ascontiguousarray(X).tobytes()).hexdigest()
        if str(z["x_sha256"]) == sha and int(z["k"]) == k:
            idx = z["idx"].astype(np.int32)
            rows = np.repeat(np.arange(X.shape[0], dtype=np.int64), k)
            d2 = oracle.pair_d2(X, rows, idx.reshape(-1)).reshape(-1, k)
            return idx, d2
    return oracle.knn(X, k)


def compare_graph(X, k, g_idx, g_d2, o_idx, o_d2, max_tie_frac=1e-3):
    """Every row of the GPU graph against the oracle's: k distinct points,
    never the row itself, float32 distances within the rounding bound of the
    exact ones, and the oracle's indices except between near-equal distances."""
    N, D = X.shape
    rtol = 2.0 * (D + 8) * 2.0 ** -24
    assert np.all(g_idx != np.arange(N)[:, None])
    s = np.sort(g_idx, 1)
    assert np.all(s[:, 1:] != s[:, :-1])
    rows = np.repeat(np.arange(N, dtype=np.int64), k)
    ex = oracle.pair_d2(X, rows, g_idx.reshape(-1)).reshape(N, k)
    np.testing.assert_allclose(g_d2, ex, rtol=rtol, atol=1e-30)
    diff = np.nonzero((g_idx != o_idx).any(1))[0]
    if diff.size:
        np.testing.assert_allclose(np.sort(ex[diff], 1), o_d2[diff], rtol=rtol, atol=1e-12)
    assert diff.size <= max(1, int(max_tie_frac * N)), diff.size
    return int(diff.size)


def check_solve(out, ref, max_label_ties=1e-4):
    Z, labels, modes, st = out
    return compare_solve(host(Z), host(labels), host(modes), st, ref, max_label_ties=max_label_ties,
                         max_mode_ties=1)


@pytest.fixture(scope="module")
def mnist_case():
    X, _ = inputs.mnist_like()
    k, L, lam = 5, 10, 1.0
    idx, d2 = oracle_graph(X, k, GOLDEN_MNIST)
    sig64 = oracle.sigma(d2, "median")
    sig = float(np.float32(sig64))   # the float32 value the C-ABI receives, on both sides
    m0 = inputs.kmeanspp(X, L, seed=1810)
    rp = np.arange(X.shape[0] + 1, dtype=np.int64) * k
    ref = oracle.solve_graph(X, L, rp, idx.reshape(-1), None, sig, lam, m0)
    return dict(X=X, k=k, L=L, lam=lam, idx=idx, d2=d2, sig=sig, sig64=sig64, m0=m0, ref=ref)


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
def test_mnist_like_full_size_solve_matches_oracle(slk, mnist_case, precision):
    c = mnist_case
    X, k, L = c["X"], c["k"], c["L"]
    Xd = dev(X)
    g = slk.knn_graph(Xd, k, precision=precision)
    compare_graph(X, k, host(g.col_idx).reshape(-1, k), host(g.dist2).reshape(-1, k),
                  c["idx"], c["d2"])
    assert slk.sigma(g.dist2, "median") == pytest.approx(c["sig64"], rel=1e-6)
    p = slk.default_params(knn_precision=precision)
    out = slk.solve(Xd, L, k, c["lam"], dev(c["m0"]), sigma=c["sig"], params=p)
    check_solve(out, c["ref"])
    ref = c["ref"]
    # the inner loops of both sides end alike: on the tolerance in the same
    # outer iterations, or on the max_inner cap (then after the same count)
    gi, oi = out[3]["inner_iters_total"], ref["inner_total"]
    assert abs(gi - oi) <= ref["outer"], (gi, oi)


@pytest.fixture(scope="module")
def manifolds_case():
    X, _ = inputs.manifolds(N=20000)
    k, L, lam = 10, 100, 1.0
    idx, d2 = oracle.knn(X, k)
    sig64 = oracle.sigma(d2, "median")
    sig = float(np.float32(sig64))
    w = oracle.heat_weights(d2.reshape(-1), sig)
    m0 = inputs.kmeanspp(X, L, seed=1810)
    rp = np.arange(X.shape[0] + 1, dtype=np.int64) * k
    ref = oracle.solve_graph(X, L, rp, idx.reshape(-1), w, sig, lam, m0)
    return dict(X=X, k=k, L=L, lam=lam, idx=idx, d2=d2, sig=sig, sig64=sig64, m0=m0, ref=ref)


def test_manifolds_subsample_solve_matches_oracle(slk, manifolds_case):
    """The precision workload's recipe at N = 20000: heat affinity, bfloat16
    tensor-core kNN candidates with the float32 rerank, 100 labels."""
    c = manifolds_case
    X, k, L = c["X"], c["k"], c["L"]
    Xd = dev(X)
    g = slk.knn_graph(Xd, k, affinity="heat", precision="bf16_rerank", sigma=c["sig"])
    compare_graph(X, k, host(g.col_idx).reshape(-1, k), host(g.dist2).reshape(-1, k),
                  c["idx"], c["d2"])
    np.testing.assert_allclose(host(g.w).reshape(-1, k),
                               oracle.heat_weights(c["d2"], c["sig"]).reshape(-1, k), rtol=1e-5)
    assert slk.sigma(g.dist2, "median") == pytest.approx(c["sig64"], rel=1e-6)
    p = slk.default_params(knn_precision="bf16_rerank", affinity="heat")
    out = slk.solve(Xd, L, k, c["lam"], dev(c["m0"]), sigma=c["sig"], params=p)
    check_solve(out, c["ref"])
    gi, oi = out[3]["inner_iters_total"], c["ref"]["inner_total"]
    assert abs(gi - oi) <= c["ref"]["outer"], (gi, oi)
