"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (float results): Z within 1e-5 max-abs, E within 1e-6 relative,
unary and sigma within 1e-6 (relative for sigma).  Integer results (kNN
indices, labels, mode indices) must be identical; where float rounding can
decide them, a difference is accepted only between near-equal candidates
(kNN: the oracle's float64 distances of the two points agree within the
float32 rounding bound of a D-term sum; labels/modes: the oracle's logits /
log z agree within 1e-5), and such near-ties are counted and bounded.
"""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Z_TOL = 1e-5
E_RTOL = 1e-6
KEY_TIE = 1e-5


@pytest.fixture(scope="module")
def slk():
    from paper_1810_13044_gb300 import build, slk as _slk
    build.build()
    return _slk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def exact_d2(X, p, qs):
    diff = X[qs].astype(np.float64) - X[p].astype(np.float64)
    return (diff * diff).sum(-1)


def check_knn(X, k, g_idx, g_d2, o_idx, o_d2, rows=None, max_tie_rows=0.01):
    """GPU rows vs oracle rows, identical up to near-equal distances."""
    N, D = X.shape
    rows = np.arange(N) if rows is None else rows
    rtol = 2.0 * (D + 8) * 2.0 ** -24
    tie_rows = 0
    for r, p in enumerate(rows):
        gi, oi = g_idx[r], o_idx[r]
        assert len(set(gi.tolist())) == k and p not in gi
        # float32 distances of the GPU are the float32 sums of the exact terms
        ex = exact_d2(X, p, gi)
        np.testing.assert_allclose(g_d2[r], ex, rtol=rtol, atol=1e-30)
        if np.array_equal(gi, oi):
            continue
        tie_rows += 1
        # only swaps among near-equal distances: the sorted exact distances agree
        np.testing.assert_allclose(np.sort(ex), o_d2[r], rtol=rtol, atol=1e-12)
    assert tie_rows <= max(1, int(max_tie_rows * len(rows))), tie_rows
    return tie_rows


# ------------------------------------------------------------------------ kNN

@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
@pytest.mark.parametrize("N,D,k,seed", [
    (2000, 16, 5, 1810),      # the 2000 x 16 blobs workload
    (2, 3, 1, 1), (3, 1, 2, 2), (17, 5, 16, 3), (129, 37, 5, 4),
    (777, 130, 24, 5), (300, 1, 5, 6), (1000, 64, 10, 7), (3000, 200, 10, 8),
])
def test_knn_matches_oracle(slk, N, D, k, seed, precision):
    if (N, D) == (2000, 16):
        X, _ = inputs.blobs(seed=seed)
    else:
        X = inputs.rng(seed).normal(size=(N, D)).astype(np.float32)
        if N > 10:
            X[N // 2] = X[1]          # an exact duplicate point
    o_idx, o_d2 = oracle.knn(X, k)
    g = slk.knn_graph(dev(X), k, precision=precision)
    g_idx = host(g.col_idx).reshape(N, k)
    g_d2 = host(g.dist2).reshape(N, k)
    np.testing.assert_array_equal(host(g.row_ptr), np.arange(N + 1) * k)
    check_knn(X, k, g_idx, g_d2, o_idx, o_d2)
    assert 0 <= g.fallback_rows <= N


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
@pytest.mark.parametrize("N,D,k,top,seed", [(2500, 8, 10, 3, 51), (4000, 12, 16, 20, 52)])
def test_knn_integer_lattice_exact_ties(slk, N, D, k, top, seed, precision):
    """Integer coordinates in [0, top]: every squared distance is a small
    integer, exact in float32 and float64, so equal distances are exact ties
    (many of them straddle the k-th place and the candidate lists' ends).
    Both sides order by (distance, index), so the graphs agree entry by
    entry, with no tie allowance."""
    X = inputs.rng(seed).integers(0, top + 1, size=(N, D)).astype(np.float32)
    o_idx, o_d2 = oracle.knn(X, k)
    g = slk.knn_graph(dev(X), k, precision=precision)
    np.testing.assert_array_equal(host(g.col_idx).reshape(N, k), o_idx)
    np.testing.assert_array_equal(host(g.dist2).reshape(N, k).astype(np.float64), o_d2)


def two_clusters(N, D, c, seed, spread=1.0):
    """Two Gaussian clusters at +-c along the first axis."""
    g = inputs.rng(seed)
    X = g.normal(0.0, spread, size=(N, D))
    X[: N // 2, 0] += c
    X[N // 2:, 0] -= c
    return X.astype(np.float32)


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
def test_knn_all_rows_through_exact_rescan(slk, precision):
    """Two tight clusters 2000 apart: the centred norms dwarf the neighbour
    distances, no row can be certified by any stage, and every row goes
    through the batched exact rescan (which must still match the oracle)."""
    N, D, k = 3000, 16, 7
    X = two_clusters(N, D, 1000.0, 31, spread=1e-2)
    o_idx, o_d2 = oracle.knn(X, k)
    gr = slk.knn_graph(dev(X), k, precision=precision)
    assert gr.fallback_rows > N // 2
    assert gr.stage_rows[2] > N // 2
    check_knn(X, k, host(gr.col_idx).reshape(N, k), host(gr.dist2).reshape(N, k), o_idx, o_d2,
              max_tie_rows=0.02)


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
@pytest.mark.parametrize("N,D,k,sample", [(2500, 1100, 10, None), (3000, 4100, 24, 150)])
def test_knn_long_rows_through_exact_rescan(slk, N, D, k, sample, precision):
    """Rows longer than the 1024 features the batched rescan keeps in
    registers go through the shared-memory rescan over (row, column range)
    items; two tight clusters far apart send every row there."""
    X = two_clusters(N, D, 1000.0, 37, spread=1e-2)
    rows = None if sample is None else np.sort(inputs.rng(38).choice(N, sample, replace=False))
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    gr = slk.knn_graph(dev(X), k, precision=precision)
    assert gr.stage_rows[2] > N // 2
    g_idx = host(gr.col_idx).reshape(N, k)
    g_d2 = host(gr.dist2).reshape(N, k)
    if rows is not None:
        g_idx, g_d2 = g_idx[rows], g_d2[rows]
    check_knn(X, k, g_idx, g_d2, o_idx, o_d2, rows=rows, max_tie_rows=0.02)


def test_knn_two_term_stage_after_bf16(slk):
    """100000 points in two unit-variance clusters 200 apart (64 dimensions;
    the two-term stage runs from 100000 points on): centred norms of about 100
    against small neighbour distances leave about a third of the rows outside
    the bfloat16 certificate (operand rounding about 2^-9 of the norm), and
    the two-term bfloat16 tiles (h + l, about 16 significant bits) certify
    nearly all of them, so hardly any row reaches the float32 stage.  Sampled
    rows against the oracle."""
    N, D, k = 100000, 64, 10
    X = two_clusters(N, D, 100.0, 61)
    gr = slk.knn_graph(dev(X), k, precision="bf16_rerank")
    open1, open2, exact = gr.stage_rows
    assert open1 == gr.fallback_rows and N // 10 < open1 < 65536, gr.stage_rows
    assert open2 <= max(8, open1 // 20), gr.stage_rows
    assert exact <= open2
    rows = np.concatenate([inputs.rng(65).choice(N, size=1200, replace=False), [0, N - 1]])
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, host(gr.col_idx).reshape(N, k)[rows], host(gr.dist2).reshape(N, k)[rows],
              o_idx, o_d2, rows=rows, max_tie_rows=0.02)


def test_knn_float32_stage_after_two_term(slk):
    """The same clusters 800 apart: the two-term tiles' accumulation bound
    (3 Dp products a dot) fails as well, and the float32 tiles with their
    certificate take the rows over."""
    N, D, k = 100000, 64, 10
    X = two_clusters(N, D, 400.0, 62)
    gr = slk.knn_graph(dev(X), k, precision="bf16_rerank")
    open1, open2, exact = gr.stage_rows
    assert open1 > N // 2 and open2 > N // 2, gr.stage_rows
    assert exact <= max(8, open2 // 20), gr.stage_rows
    rows = np.concatenate([inputs.rng(66).choice(N, size=1200, replace=False), [0, N - 1]])
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, host(gr.col_idx).reshape(N, k)[rows], host(gr.dist2).reshape(N, k)[rows],
              o_idx, o_d2, rows=rows, max_tie_rows=0.02)


def test_knn_small_graph_skips_two_term_stage(slk):
    """Below 100000 points the rows the bfloat16 certificate leaves open go
    straight to the float32 stage (4000 points, clusters 400 apart)."""
    N, D, k = 4000, 64, 10
    X = two_clusters(N, D, 200.0, 61)
    o_idx, o_d2 = oracle.knn(X, k)
    gr = slk.knn_graph(dev(X), k, precision="bf16_rerank")
    open1, open2, exact = gr.stage_rows
    assert open1 > N // 2 and open2 == open1, gr.stage_rows
    assert exact <= max(8, open2 // 20), gr.stage_rows
    check_knn(X, k, host(gr.col_idx).reshape(N, k), host(gr.dist2).reshape(N, k), o_idx, o_d2,
              max_tie_rows=0.02)


def test_knn_two_term_stage_capacity(slk):
    """150000 points in two clusters 140 apart (16 dimensions): more than
    65536 rows fail the bfloat16 certificate; the two-term stage takes the
    first 65536 of them and passes the rest straight to the float32 stage,
    so that stage receives at least the excess.  Sampled rows against the
    oracle."""
    N, D, k = 150000, 16, 10
    X = two_clusters(N, D, 70.0, 63)
    gr = slk.knn_graph(dev(X), k, precision="bf16_rerank")
    open1, open2, exact = gr.stage_rows
    cap = 65536
    assert open1 > cap, gr.stage_rows
    assert open1 - cap <= open2 <= open1 - cap + cap // 50, gr.stage_rows
    rows = inputs.rng(64).choice(N, size=1500, replace=False)
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, host(gr.col_idx).reshape(N, k)[rows], host(gr.dist2).reshape(N, k)[rows],
              o_idx, o_d2, rows=rows, max_tie_rows=0.02)


@pytest.mark.parametrize("D", [32, 130])
def test_knn_float32_stage_after_bf16(slk, D):
    """Clusters far from the data mean (centred norms ~ 900 with unit
    neighbour distances): neither the bfloat16 nor the two-term certificate
    can hold, the float32 query tiles and their certificate take the rows
    over, and the graph still matches the oracle on every row."""
    g = inputs.rng(41 + D)
    N, k = 1500, 7
    c = g.normal(0.0, 30.0, size=(3, D))
    X = (c[g.integers(0, 3, N)] + g.normal(0.0, 0.5, size=(N, D))).astype(np.float32)
    o_idx, o_d2 = oracle.knn(X, k)
    gr = slk.knn_graph(dev(X), k, precision="bf16_rerank")
    assert gr.fallback_rows > N // 10
    assert gr.stage_rows[1] > 0
    check_knn(X, k, host(gr.col_idx).reshape(N, k), host(gr.dist2).reshape(N, k), o_idx, o_d2,
              max_tie_rows=0.02)


def test_knn_heat_weights(slk):
    X, _ = inputs.blobs(N=500, D=6, n_blobs=3, seed=9)
    o_idx, o_d2 = oracle.knn(X, 5)
    sig = 1.7
    g = slk.knn_graph(dev(X), 5, affinity="heat", sigma=sig)
    w = host(g.w)
    np.testing.assert_allclose(w, np.exp(-host(g.dist2).astype(np.float64) / (2 * sig * sig)),
                               rtol=2e-6)
    np.testing.assert_allclose(np.sort(w.reshape(500, 5), 1),
                               np.sort(oracle.heat_weights(o_d2, sig).reshape(500, 5), 1), rtol=1e-5)


def test_knn_mnist_like_full_size_sampled(slk):
    """70000 x 784, k = 5 (the scale workload), sampled rows vs the oracle;
    the bfloat16 tensor-core candidates give the same graph as the float32
    ones (both equal a full float32 scan once certified or rescanned)."""
    X, _ = inputs.mnist_like()
    k = 5
    Xd = dev(X)
    g = slk.knn_graph(Xd, k)
    g_idx = host(g.col_idx).reshape(-1, k)
    g_d2 = host(g.dist2).reshape(-1, k)
    rows = inputs.rng(99).choice(X.shape[0], size=24, replace=False)
    rows = np.concatenate([rows, [0, X.shape[0] - 1]])
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, g_idx[rows], g_d2[rows], o_idx, o_d2, rows=rows, max_tie_rows=0.1)
    assert g.fallback_rows < X.shape[0] * 0.05
    gb = slk.knn_graph(Xd, k, precision="bf16_rerank")
    np.testing.assert_array_equal(host(gb.col_idx), host(g.col_idx))
    np.testing.assert_array_equal(host(gb.dist2), host(g.dist2))
    assert gb.fallback_rows < X.shape[0] * 0.05


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
def test_knn_single_column_split_sampled(slk, precision):
    """N = 19456 = 152 x 128: one work item per row block on 152 SMs, so every
    row has a single candidate list (the tensor-core list keeps the row's own
    column, which the rerank drops)."""
    X = inputs.rng(21).normal(size=(19456, 40)).astype(np.float32)
    k = 10
    g = slk.knn_graph(dev(X), k, precision=precision)
    rows = inputs.rng(22).choice(X.shape[0], size=64, replace=False)
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, host(g.col_idx).reshape(-1, k)[rows], host(g.dist2).reshape(-1, k)[rows],
              o_idx, o_d2, rows=rows, max_tie_rows=0.05)


def test_knn_manifolds_full_size_sampled(slk):
    """The precision workload: 1e6 x 128, k = 10, heat weights, bfloat16
    tensor-core candidates with the float32 rerank; sampled rows vs the oracle."""
    X, _ = inputs.manifolds()
    k = 10
    g = slk.knn_graph(dev(X), k, affinity="heat", precision="bf16_rerank", sigma=2.0)
    rows = inputs.rng(23).choice(X.shape[0], size=12, replace=False)
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, host(g.col_idx).reshape(-1, k)[rows], host(g.dist2).reshape(-1, k)[rows],
              o_idx, o_d2, rows=rows, max_tie_rows=0.25)
    w = host(g.w).reshape(-1, k)[rows]
    np.testing.assert_allclose(w, np.exp(-host(g.dist2).reshape(-1, k)[rows].astype(np.float64) / 8.0),
                               rtol=2e-6)
    assert g.fallback_rows < X.shape[0] * 0.05


# ---------------------------------------------------------------------- sigma

@pytest.mark.parametrize("n", [1, 2, 5, 10000, 10001])
@pytest.mark.parametrize("rule", ["median", "meansq"])
def test_sigma_matches_oracle(slk, n, rule):
    d2 = inputs.rng(n).uniform(0.01, 30.0, size=n).astype(np.float32)
    if n > 4:
        d2[: n // 3] = d2[0]           # many exact ties
    got = slk.sigma(dev(d2), rule)
    want = oracle.sigma(d2.astype(np.float64), rule)
    assert got == pytest.approx(want, rel=1e-6)


# ---------------------------------------------------------------------- unary

@pytest.mark.parametrize("N,D,L", [(2000, 16, 5), (70, 1, 1), (333, 31, 33), (500, 784, 10),
                                   (257, 128, 100), (300, 7, 256)])
def test_unary_matches_oracle(slk, N, D, L):
    g = inputs.rng(N + D + L)
    X = g.normal(size=(N, D)).astype(np.float32)
    modes = g.choice(N, size=L, replace=False).astype(np.int32)
    d2 = oracle.knn(X[:50], 3)[1]
    sig = float(np.sqrt(np.median(d2)) * 1.5)
    A, Z0 = slk.unary(dev(X), dev(modes), sig)
    Ao = oracle.unary(X, modes, sig)
    assert np.abs(host(A) - Ao).max() <= 1e-6
    assert np.abs(host(Z0) - oracle.softmax_rows(Ao)).max() <= 1e-6


# --------------------------------------------------------------- bound iterate

BOUND_CASES = [(1000, 5, 5, False), (1000, 1, 3, False), (1001, 2, 5, True), (2000, 10, 5, False),
               (777, 17, 7, True), (500, 33, 4, False), (400, 100, 10, True), (300, 256, 5, False),
               (5, 3, 4, False), (2, 2, 1, True)]


def _bound_inputs(N, L, k, weighted, seed):
    rp, ci, w = inputs.random_graph(N, k, seed=seed, weighted=weighted)
    A = inputs.random_unary(N, L, seed=seed + 1)
    Z0 = inputs.random_simplex_rows(N, L, seed=seed + 2)
    return rp, ci, w, A, Z0


@pytest.mark.parametrize("N,L,k,weighted", BOUND_CASES)
def test_bound_iterate_fixed_iterations(slk, N, L, k, weighted):
    rp, ci, w, A, Z0 = _bound_inputs(N, L, k, weighted, seed=N * 7 + L)
    lam = 1.3
    for iters in (1, 2, 7):
        Z, Zp = dev(Z0), torch.empty_like(dev(Z0))
        it, dl = slk.bound_iterate(dev(A), dev(rp), dev(ci), None if w is None else dev(w), lam,
                                   Z, Zp, iters, tol=-1.0)
        Zo, Zpo, ito, dlo = oracle.bound_iterate(A, rp, ci, w, lam, Z0, iters)
        assert it == ito == iters
        assert np.abs(host(Z) - Zo).max() <= Z_TOL
        assert np.abs(host(Zp) - Zpo).max() <= Z_TOL
        assert dl == pytest.approx(dlo, abs=2 * Z_TOL)
        np.testing.assert_allclose(host(Z).sum(1), 1.0, atol=1e-5)


@pytest.mark.parametrize("N,L,k", [(3000, 5, 5), (2000, 12, 6)])
def test_bound_iterate_until_converged(slk, N, L, k):
    rp, ci, w, A, Z0 = _bound_inputs(N, L, k, False, seed=5)
    lam, tol = 1.0, 1e-6
    Z, Zp = dev(Z0), torch.empty_like(dev(Z0))
    it, dl = slk.bound_iterate(dev(A), dev(rp), dev(ci), None, lam, Z, Zp, 100, tol=tol)
    Zo, _, ito, _ = oracle.bound_iterate(A, rp, ci, None, lam, Z0, 100, tol=tol)
    assert abs(it - ito) <= 1 and it < 100
    assert dl <= tol
    assert np.abs(host(Z) - Zo).max() <= Z_TOL


@pytest.mark.parametrize("N,L,k,iters", [(70000, 10, 5, 3), (200000, 100, 10, 2)])
def test_bound_iterate_full_size(slk, N, L, k, iters):
    """The bound-iteration shapes of the 70000 x 784 (L=10, k=5) and
    1e6 x 128 (L=100, k=10; 2e5 rows here) workloads."""
    rp, ci, w, A, Z0 = _bound_inputs(N, L, k, L == 100, seed=11)
    Z, Zp = dev(Z0), torch.empty_like(dev(Z0))
    it, _ = slk.bound_iterate(dev(A), dev(rp), dev(ci), None if w is None else dev(w), 1.0, Z, Zp,
                              iters, tol=-1.0)
    Zo, _, _, _ = oracle.bound_iterate(A, rp, ci, w, 1.0, Z0, iters)
    assert it == iters
    assert np.abs(host(Z) - Zo).max() <= Z_TOL


# ----------------------------------------------------------------- mode update

def _near_tie_modes(g_modes, o_modes, logZ):
    bad = []
    for l, (gq, oq) in enumerate(zip(g_modes, o_modes)):
        if gq != oq and abs(logZ[gq, l] - logZ[oq, l]) > KEY_TIE:
            bad.append((l, gq, oq, logZ[gq, l], logZ[oq, l]))
    return bad


@pytest.mark.parametrize("N,L,k,weighted", BOUND_CASES[:8])
def test_mode_update_matches_oracle(slk, N, L, k, weighted):
    rp, ci, w, A, Z0 = _bound_inputs(N, L, k, weighted, seed=N + 3 * L)
    lam = 2.0
    Zp_in = dev(Z0)
    modes = dev(np.zeros(L, np.int32))
    changed, labels, key = slk.mode_update(dev(A), Zp_in, dev(rp), dev(ci),
                                           None if w is None else dev(w), lam, modes)
    S = oracle.logits(A, rp, ci, w, lam, Z0)
    om, okey = oracle.mode_update(S)
    logZ = oracle.log_z(S)
    assert not _near_tie_modes(host(modes), om, logZ)
    assert np.abs(host(key) - okey).max() <= KEY_TIE
    ol = oracle.labels(S)
    gl = host(labels)
    diff = np.nonzero(gl != ol)[0]
    for p in diff:
        assert abs(S[p, gl[p]] - S[p, ol[p]]) <= KEY_TIE
    assert changed == int(not np.array_equal(om, np.zeros(L)))
    # without Z_prev the logits are A itself
    modes2 = dev(np.zeros(L, np.int32))
    slk.mode_update(dev(A), None, dev(rp), dev(ci), None, lam, modes2)
    om2, _ = oracle.mode_update(A.astype(np.float64))
    assert not _near_tie_modes(host(modes2), om2, oracle.log_z(A.astype(np.float64)))


def test_mode_update_saturated_logits(slk):
    """Logit gaps of 40: float32 z rounds to 1.0, the log1p key still orders points."""
    N, L = 64, 3
    A = np.zeros((N, L), np.float32)
    A[:, 0] = 20.0 + np.arange(N, dtype=np.float32) * 0.25   # later points more confident
    A[:, 1] = -20.0
    rp, ci, _ = inputs.random_graph(N, 2, seed=1)
    modes = dev(np.zeros(L, np.int32))
    slk.mode_update(dev(A), None, dev(rp), dev(ci), None, 1.0, modes)
    om, _ = oracle.mode_update(A.astype(np.float64))
    assert host(modes)[0] == om[0] == N - 1


# ---------------------------------------------------------------------- energy

@pytest.mark.parametrize("weighted", [False, True])
def test_energy_matches_oracle(slk, weighted):
    X, _ = inputs.blobs(N=2000, D=16, seed=4)
    N, L = X.shape[0], 5
    rp, ci, w = inputs.random_graph(N, 5, seed=8, weighted=weighted)
    lab = inputs.rng(3).integers(0, L, size=N).astype(np.int32)
    modes = np.array([1, 100, 200, 300, 1999], np.int32)
    sig, lam = 2.5, 1.5
    E = slk.energy(dev(X), dev(lab), dev(rp), dev(ci), None if w is None else dev(w), L, dev(modes),
                   sig, lam)
    Eo = oracle.energy(X, lab, rp, ci, w, L, modes, np.float64(np.float32(sig)), np.float32(lam))
    assert E == pytest.approx(Eo, rel=E_RTOL)


# ----------------------------------------------------------------- whole solve

def _compare_solve(out_gpu, ref, X):
    Z, labels, modes, stats = out_gpu
    assert stats["outer_iters"] == ref["outer"]
    np.testing.assert_array_equal(host(modes), ref["modes"])
    np.testing.assert_array_equal(host(labels), ref["labels"])
    assert np.abs(host(Z) - ref["Z"]).max() <= Z_TOL
    assert stats["energy"] == pytest.approx(ref["E"], rel=E_RTOL)


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
def test_solve_blobs_matches_oracle(slk, precision):
    """2000 x 16 blobs, L=5, k=5, lambda=1, sigma = median kNN distance."""
    X, _ = inputs.blobs()
    L, k, lam = 5, 5, 1.0
    m0 = inputs.kmeanspp(X, L, seed=1810)
    ref = oracle.solve(X, L, k, lam, m0)
    p = slk.default_params(knn_precision=precision)
    out = slk.solve(dev(X), L, k, lam, dev(m0), params=p)
    assert out[3]["sigma"] == pytest.approx(ref["sigma"], rel=1e-6)
    # the run is then repeated with the oracle's sigma so that both start equal
    out = slk.solve(dev(X), L, k, lam, dev(m0), sigma=ref["sigma"], params=p)
    _compare_solve(out, ref, X)
    assert out[3]["converged"] == 1


@pytest.mark.parametrize("seed", [3, 4])
def test_solve_multi_outer_matches_oracle(slk, seed):
    """Overlapping blobs and a bad seed so that the modes move over several
    outer iterations."""
    X, _ = inputs.blobs(N=1500, D=4, n_blobs=6, centre_var=6.0, seed=seed)
    L, k, lam = 6, 5, 2.0
    m0 = np.arange(L, dtype=np.int32)
    ref = oracle.solve(X, L, k, lam, m0)
    out = slk.solve(dev(X), L, k, lam, dev(m0), sigma=ref["sigma"])
    _compare_solve(out, ref, X)


def test_solve_heat_affinity_and_meansq_sigma(slk):
    X, _ = inputs.manifolds(N=3000, D=32, n_clusters=6, seed=5)
    L, k, lam = 6, 10, 1.0
    m0 = inputs.kmeanspp(X, L, seed=5)
    idx, d2 = oracle.knn(X, k)
    sig = oracle.sigma(d2, "meansq")
    rp = np.arange(X.shape[0] + 1, dtype=np.int64) * k
    w = oracle.heat_weights(d2.reshape(-1), sig)
    ref = oracle.solve_graph(X, L, rp, idx.reshape(-1), w, sig, lam, m0)
    p = slk.default_params(affinity="heat", sigma_rule="meansq")
    out = slk.solve(dev(X), L, k, lam, dev(m0), params=p)
    assert out[3]["sigma"] == pytest.approx(sig, rel=1e-6)
    # weights come from float32 distances: compare within the Z tolerance
    out = slk.solve(dev(X), L, k, lam, dev(m0), sigma=sig, params=p)
    Z, labels, modes, stats = out
    np.testing.assert_array_equal(host(modes), ref["modes"])
    np.testing.assert_array_equal(host(labels), ref["labels"])
    assert np.abs(host(Z) - ref["Z"]).max() <= Z_TOL
    assert stats["energy"] == pytest.approx(ref["E"], rel=E_RTOL)


@pytest.mark.parametrize("case", ["blobs", "multi_outer", "heat"])
def test_solve_sorted_row_order_is_identical(slk, case):
    """The z-updates on rows sorted by their nearest initial mode (reorder)
    give the same bits as the given order: each row keeps its edge order and
    mode ties go to the smaller original index."""
    if case == "blobs":
        X, _ = inputs.blobs()
        L, k, lam, m0, aff = 5, 5, 1.0, inputs.kmeanspp(inputs.blobs()[0], 5, seed=1810), "binary"
    elif case == "multi_outer":
        X, _ = inputs.blobs(N=1500, D=4, n_blobs=6, centre_var=6.0, seed=4)
        L, k, lam, m0, aff = 6, 5, 2.0, np.arange(6, dtype=np.int32), "binary"
    else:
        X, _ = inputs.manifolds(N=3000, D=32, n_clusters=6, seed=5)
        L, k, lam, m0, aff = 6, 10, 1.0, inputs.kmeanspp(X, 6, seed=5), "heat"
    outs = []
    for ro in (0, 1):
        p = slk.default_params(affinity=aff, reorder=ro)
        outs.append(slk.solve(dev(X), L, k, lam, dev(m0), params=p))
    (Z0, l0, m0_, s0), (Z1, l1, m1, s1) = outs
    assert torch.equal(Z0, Z1) and torch.equal(l0, l1) and torch.equal(m0_, m1)
    assert s0["outer_iters"] == s1["outer_iters"] and s0["inner_iters_total"] == s1["inner_iters_total"]
    assert s1["energy"] == pytest.approx(s0["energy"], rel=1e-12)


def test_solve_mnist_like_full_size(slk):
    """The 70000 x 784, L=10, k=5 workload in the launch configuration the
    benchmark times.  The oracle checks sampled kNN rows; the rest is checked
    through properties that hold at any size."""
    X, _ = inputs.mnist_like()
    L, k, lam = 10, 5, 1.0
    m0 = inputs.kmeanspp(X, L, seed=1810)
    Xd = dev(X)
    Z, labels, modes, st = slk.solve(Xd, L, k, lam, dev(m0))
    Zh = host(Z).astype(np.float64)
    np.testing.assert_allclose(Zh.sum(1), 1.0, atol=1e-5)
    assert np.all(Zh > 0)
    m = host(modes)
    assert np.all((m >= 0) & (m < X.shape[0]))
    lab = host(labels)
    srt = np.sort(Zh, 1)
    clear = srt[:, -1] - srt[:, -2] > 1e-6          # rows without a float32 near-tie
    np.testing.assert_array_equal(lab[clear], np.argmax(Zh, 1)[clear])
    # each mode holds the largest z of its column (up to float32 near-ties)
    for l in range(L):
        assert Zh[m[l], l] >= Zh[:, l].max() - 1e-6
    # the energy is the library's own Eq. (1) on the returned labels/modes
    g = slk.knn_graph(Xd, k)
    E = slk.energy(Xd, labels, g.row_ptr, g.col_idx, None, L, modes, st["sigma"], lam)
    assert E == pytest.approx(st["energy"], rel=1e-12)
    # sampled kNN rows of this graph vs the oracle
    rows = inputs.rng(5).choice(X.shape[0], size=8, replace=False)
    o_idx, o_d2 = oracle.knn(X, k, rows=rows)
    check_knn(X, k, host(g.col_idx).reshape(-1, k)[rows], host(g.dist2).reshape(-1, k)[rows],
              o_idx, o_d2, rows=rows, max_tie_rows=0.25)
    # the host-buffer entry point gives the same result
    Zh2, lab2, m2, st2 = slk.solve_host(torch.from_numpy(X).pin_memory(), L, k, lam,
                                        torch.from_numpy(m0), want_z=True)
    np.testing.assert_array_equal(lab2.numpy(), lab)
    np.testing.assert_array_equal(m2.numpy(), m)
    assert np.abs(Zh2.numpy() - host(Z)).max() == 0.0
    assert st2["energy"] == pytest.approx(st["energy"], rel=1e-12)


def test_host_solve_profiles_its_transfers(slk):
    """The host-buffer solve records its copies as the transfer phase (one
    scope for the copies in, one for the copies out); the device solve has
    none."""
    X, _ = inputs.blobs(seed=1810)
    L, k, lam = 5, 5, 1.0
    m0 = np.arange(L, dtype=np.int32) * 7
    ctx = slk.context(0)
    ctx.profile(True)
    slk.solve_host(torch.from_numpy(X).pin_memory(), L, k, lam, torch.from_numpy(m0), ctx=ctx)
    ms, calls, _ = ctx.profile_read()
    ctx.profile(False)
    assert calls["transfer"] == 2 and ms["transfer"] > 0.0
    assert calls["knn_cand"] >= 1
    ctx.profile(True)
    slk.solve(dev(X), L, k, lam, dev(m0), ctx=ctx)
    ms, calls, _ = ctx.profile_read()
    ctx.profile(False)
    assert calls["transfer"] == 0


# --------------------------------------------------------------- bad arguments

def test_invalid_arguments_are_rejected(slk):
    X = dev(inputs.rng(0).normal(size=(10, 3)).astype(np.float32))
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.knn_graph(X, 10)                      # k > N - 1
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.unary(X, dev(np.arange(11, dtype=np.int32)), 1.0)   # L > N
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.unary(X, dev(np.arange(3, dtype=np.int32)), -1.0)   # sigma <= 0
    A = dev(np.ones((10, 3), np.float32))
    Z = dev(np.full((10, 3), 1 / 3, np.float32))
    rp, ci, _ = inputs.random_graph(10, 2, seed=0)
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.bound_iterate(A, dev(rp), dev(ci), None, 1.0, Z, Z, 3)  # aliasing buffers
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.solve(X, 3, 2, 1.0, dev(np.arange(3, dtype=np.int32)),
                  params=slk.default_params(max_inner=0))
