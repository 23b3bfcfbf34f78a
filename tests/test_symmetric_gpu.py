"""The symmetric affinity (K + K^t) / 2 (Prop. 1 assumes a symmetric K) on
the GPU: slk_symmetrize against the oracle's, and whole solves on it
(slk_params.symmetrize) against the oracle's solve on its own symmetrised
exact kNN graph."""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs
from parity_checks import compare_solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slk():
    from paper_1810_13044_gb300 import build, slk as _slk
    build.build()
    return _slk


def dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("N,k,weighted", [(2, 1, False), (50, 4, False), (3001, 7, True),
                                          (20000, 10, True), (5000, 24, False)])
def test_symmetrize_matches_oracle(slk, N, k, weighted):
    rp, ci, w = inputs.random_graph(N, k, seed=N + 3 * k, weighted=weighted)
    g_rp, g_ci, g_w = slk.symmetrize(dev(rp), dev(ci), dev(w), N)
    o_rp, o_ci, o_w = oracle.symmetrize(rp, ci, w, N)
    np.testing.assert_array_equal(g_rp.cpu().numpy(), o_rp)
    np.testing.assert_array_equal(g_ci.cpu().numpy(), o_ci)
    np.testing.assert_allclose(g_w.cpu().numpy(), o_w, rtol=2 ** -23, atol=0)


def test_symmetrize_of_a_knn_graph_with_hubs(slk):
    """A kNN graph of clustered points (many points list the same hub):
    long in-lists, mutual edges merged."""
    X, _ = inputs.mixture(6000, 9, 4, seed=3)
    g = slk.knn_graph(dev(X), 10)
    rp, ci = g.row_ptr.cpu().numpy(), g.col_idx.cpu().numpy()
    g_rp, g_ci, g_w = slk.symmetrize(g.row_ptr, g.col_idx, None, X.shape[0])
    o_rp, o_ci, o_w = oracle.symmetrize(rp, ci, None, X.shape[0])
    np.testing.assert_array_equal(g_rp.cpu().numpy(), o_rp)
    np.testing.assert_array_equal(g_ci.cpu().numpy(), o_ci)
    np.testing.assert_array_equal(g_w.cpu().numpy(), o_w.astype(np.float32))


def test_symmetrize_rejects_long_rows(slk):
    N = 40
    rp = np.array([0, 30] + [30] * (N - 1), np.int64)
    ci = np.arange(1, 31, dtype=np.int32)
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.symmetrize(dev(rp), dev(ci), None, N)


@pytest.mark.parametrize("case", ["blobs", "heat", "multi_outer"])
def test_solve_on_symmetric_affinity_matches_oracle(slk, case):
    if case == "blobs":
        X, _ = inputs.blobs()
        L, k, lam, aff = 5, 5, 1.0, "binary"
        m0 = inputs.kmeanspp(X, L, seed=1810)
    elif case == "heat":
        X, _ = inputs.manifolds(N=3000, D=32, n_clusters=6, seed=5)
        L, k, lam, aff = 6, 10, 1.0, "heat"
        m0 = inputs.kmeanspp(X, L, seed=5)
    else:
        X, _ = inputs.blobs(N=1500, D=4, n_blobs=6, centre_var=6.0, seed=3)
        L, k, lam, aff = 6, 5, 2.0, "binary"
        m0 = np.arange(L, dtype=np.int32)
    # both sides take the kernel width as the float32 value the C-ABI receives
    sig = float(np.float32(oracle.sigma(oracle.knn(X, k)[1], "median")))
    ref = oracle.solve(X, L, k, lam, m0, affinity=aff, sig=sig, symmetric=True)
    p = slk.default_params(affinity=aff, symmetrize=1)
    Z, lab, modes, st = slk.solve(dev(X), L, k, lam, dev(m0), sigma=ref["sigma"], params=p)
    compare_solve(Z.cpu().numpy(), lab.cpu().numpy(), modes.cpu().numpy(), st, ref,
                  max_label_ties=1e-3, max_mode_ties=0)
    # and it differs from the directed solve (the option is not a no-op)
    Zd, _, _, _ = slk.solve(dev(X), L, k, lam, dev(m0), sigma=ref["sigma"],
                            params=slk.default_params(affinity=aff))
    assert (Zd - Z).abs().max().item() > 1e-4


def test_batched_and_server_refuse_symmetrize(slk):
    X, _ = inputs.blobs(N=300, D=4, n_blobs=3, seed=1)
    pr = dict(X=dev(X), L=3, k=5, lam=1.0, init_modes=dev(np.array([0, 1, 2], np.int32)))
    p = slk.default_params(symmetrize=1)
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.solve_batched([pr], params=p)
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.Server(max_slots=2, quantum=2, memory_bytes=64 << 20, params=p)
