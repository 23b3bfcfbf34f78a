"""Pins of the FP64 oracle to things other than itself.

Each test checks one oracle function against what the paper and the
mathematics fix: brute force on tiny inputs, closed forms, library special
cases, invariants (simplex rows, the auxiliary-function descent of Section 3,
the Laplacian identity of Eq. 3).  Each is chosen so that a plausible mistake
(a dropped term, a wrong sign or factor, a transposed operand, a wrong
tie-break) fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy.special import log_softmax, softmax

import oracle
from paper_1810_13044_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- kNN (Section 4.2)

def _knn_brute(X, k):
    """Full distance matrix + full lexicographic sort (numpy), self excluded."""
    X = X.astype(np.float64)
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    N = X.shape[0]
    idx = np.empty((N, k), np.int64)
    for p in range(N):
        q = np.array([j for j in range(N) if j != p])
        order = np.lexsort((q, D2[p, q]))
        idx[p] = q[order[:k]]
    return idx, D2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_knn_matches_full_sort_with_ties(seed):
    g = inputs.rng(seed)
    # integer grid points: many exactly tied distances, and duplicated points
    X = g.integers(0, 4, size=(60, 3)).astype(np.float32)
    X[10] = X[3]
    X[11] = X[3]
    k = 7
    idx, d2 = oracle.knn(X, k)
    ref, D2 = _knn_brute(X, k)
    np.testing.assert_array_equal(idx, ref)
    np.testing.assert_array_equal(d2, np.take_along_axis(D2, ref, 1))
    # duplicates are ordinary neighbours at distance 0
    assert 10 in idx[3] and 11 in idx[3] and d2[3, 0] == 0.0


def test_knn_excludes_self_and_full_neighbourhood():
    X = inputs.rng(5).normal(size=(9, 4)).astype(np.float32)
    idx, d2 = oracle.knn(X, 8)         # k = N - 1: every other point, sorted
    for p in range(9):
        assert p not in idx[p]
        assert sorted(idx[p].tolist()) == [q for q in range(9) if q != p]
        assert np.all(np.diff(d2[p]) >= 0)
    with pytest.raises(ValueError):
        oracle.knn(X, 9)


def test_knn_rows_subset_equals_full():
    X = inputs.rng(7).normal(size=(200, 5)).astype(np.float32)
    full_i, full_d = oracle.knn(X, 5)
    rows = np.array([0, 17, 199, 42])
    i, d = oracle.knn(X, 5, rows=rows)
    np.testing.assert_array_equal(i, full_i[rows])
    np.testing.assert_array_equal(d, full_d[rows])


# --------------------------------------------------------------------------- sigma (Section 4.2)

@pytest.mark.parametrize("n", [1, 2, 7, 10])
def test_sigma_median_and_meansq(n):
    d2 = inputs.rng(n).uniform(0.1, 9.0, size=n)
    assert oracle.sigma(d2, "median") == pytest.approx(np.median(np.sqrt(d2)), rel=1e-15)
    assert oracle.sigma(d2, "meansq") == pytest.approx(math.sqrt(np.mean(d2)), rel=1e-14)


# --------------------------------------------------------------------------- unary (Eq. general-second)

def test_unary_closed_form():
    X = np.array([[0.0], [1.0], [3.0], [-2.0]], np.float32)
    A = oracle.unary(X, [0, 2], 1.5)
    # k(x, y) = exp(-(x - y)^2 / (2 sigma^2)), sigma^2 = 2.25
    want = np.array([[1.0, math.exp(-9 / 4.5)],
                     [math.exp(-1 / 4.5), math.exp(-4 / 4.5)],
                     [math.exp(-9 / 4.5), 1.0],
                     [math.exp(-4 / 4.5), math.exp(-25 / 4.5)]])
    np.testing.assert_allclose(A, want, rtol=1e-15)


def test_unary_mode_is_one_and_range():
    X, _ = inputs.blobs(N=300, D=6, n_blobs=3, seed=3)
    modes = inputs.kmeanspp(X, 3, seed=3)
    A = oracle.unary(X, modes, 2.0)
    for l, m in enumerate(modes):
        assert A[m, l] == 1.0
    assert np.all(A > 0) and np.all(A <= 1)


# --------------------------------------------------------------------------- z-update (Eq. soft-max)

def _aux_value(z, a, lb):
    with np.errstate(divide="ignore", invalid="ignore"):
        ent = np.where(z > 0, z * np.log(z), 0.0).sum(-1)
    return ent - (z * (a + lb)).sum(-1)


@pytest.mark.parametrize("L", [2, 3])
def test_update_minimises_per_point_subproblem(L):
    """Eq. (AUX-Form): z_p^{i+1} minimises z^t (log z - a_p - lambda b_p) over
    the simplex.  Brute force over a fine simplex grid; b_p is built through a
    weighted two-node graph so the whole update (pairwise term, lambda, sign)
    is exercised."""
    g = inputs.rng(10 + L)
    a0 = g.uniform(0, 1, size=L)
    z1 = g.dirichlet(np.ones(L))
    lam, w01 = 1.7, 0.6
    A = np.stack([a0, g.uniform(0, 1, size=L)])
    Z0 = np.stack([g.dirichlet(np.ones(L)), z1])
    row_ptr = np.array([0, 1, 2])
    col = np.array([1, 0])
    w = np.array([w01, 0.3])
    Z, _, it, _ = oracle.bound_iterate(A, row_ptr, col, w, lam, Z0, 1)
    assert it == 1
    zo = Z[0]
    h = 1.0 / 600
    if L == 2:
        t = np.arange(0, 1 + h / 2, h)
        grid = np.stack([t, 1 - t], -1)
    else:
        pts = [(i * h, j * h) for i in range(601) for j in range(601 - i)]
        u = np.array(pts)
        grid = np.stack([u[:, 0], u[:, 1], np.clip(1 - u[:, 0] - u[:, 1], 0, 1)], -1)
    vals = _aux_value(grid, a0, lam * w01 * z1)
    best = grid[np.argmin(vals)]
    assert np.max(np.abs(best - zo)) < 2.5 * h
    assert _aux_value(zo[None], a0, lam * w01 * z1)[0] <= vals.min() + 1e-12
    # and not the update with the pairwise sign flipped or lambda dropped
    wrong = softmax(a0 - lam * w01 * z1)
    assert np.max(np.abs(wrong - zo)) > 1e-3 or np.allclose(z1, z1.mean())


def test_pairwise_is_row_times_Z_dense():
    """b = K Z with K taken row-wise (not K^T): dense matmul on a
    non-symmetric weighted graph."""
    N, k, L = 50, 4, 3
    rp, ci, w = inputs.random_graph(N, k, seed=4, weighted=True)
    Z = inputs.random_simplex_rows(N, L, seed=5).astype(np.float64)
    K = np.zeros((N, N))
    for p in range(N):
        for e in range(rp[p], rp[p + 1]):
            K[p, ci[e]] += w[e]
    assert not np.allclose(K, K.T)
    np.testing.assert_allclose(oracle.pairwise(rp, ci, w.astype(np.float64), Z), K @ Z, rtol=1e-13)
    # binary weights when w is None
    Kb = (K > 0).astype(np.float64)
    np.testing.assert_allclose(oracle.pairwise(rp, ci, None, Z), Kb @ Z, rtol=1e-13)


def test_lambda_zero_and_single_label():
    N, k, L = 40, 3, 4
    rp, ci, _ = inputs.random_graph(N, k, seed=6)
    A = inputs.random_unary(N, L, seed=7).astype(np.float64)
    Z0 = inputs.random_simplex_rows(N, L, seed=8).astype(np.float64)
    Z, _, it, _ = oracle.bound_iterate(A, rp, ci, None, 0.0, Z0, 5)
    np.testing.assert_allclose(Z, softmax(A, axis=1), rtol=1e-14)
    assert it == 5
    # lambda = 0: the first update lands on softmax(A), the second changes
    # nothing, so a tolerance-0 run stops after exactly two updates
    Z, _, it, dl = oracle.bound_iterate(A, rp, ci, None, 0.0, Z0, 50, tol=0.0)
    assert (it, dl) == (2, 0.0)
    Z1, _, _, _ = oracle.bound_iterate(A[:, :1], rp, ci, None, 2.0, np.ones((N, 1)), 3)
    np.testing.assert_array_equal(Z1, np.ones((N, 1)))


def test_rows_on_simplex_and_convergence_stop():
    N, k, L = 300, 5, 6
    rp, ci, _ = inputs.random_graph(N, k, seed=9)
    A = inputs.random_unary(N, L, seed=10).astype(np.float64)
    Z0 = softmax(A, axis=1)
    Z, Zp, it, dl = oracle.bound_iterate(A, rp, ci, None, 1.0, Z0, 200, tol=1e-9)
    assert it < 200 and dl <= 1e-9
    assert np.max(np.abs(Z - Zp)) == pytest.approx(dl, abs=0)
    np.testing.assert_allclose(Z.sum(1), 1.0, atol=1e-14)
    assert np.all(Z > 0)


def _dense_csr(K):
    N = K.shape[0]
    rp = np.arange(N + 1, dtype=np.int64) * N
    ci = np.tile(np.arange(N, dtype=np.int32), N)
    return rp, ci, K.reshape(-1).copy()


def test_relaxed_objective_descends_with_psd_kernel():
    """Section 3 / Prop. 1: with a symmetric psd affinity the soft-max update
    minimises an auxiliary function of the relaxation, so the relaxed
    objective never increases.  The update z ~ exp(a + lambda K z) is the exact
    minimiser of the bound of R with lambda/2 on its pairwise term (the
    gradient of the quadratic form z^t K z is 2 K z)."""
    X, _ = inputs.blobs(N=40, D=3, n_blobs=3, centre_var=4.0, seed=11)
    D2 = ((X[:, None].astype(np.float64) - X[None]) ** 2).sum(-1)
    K = np.exp(-D2 / 2.0)                  # Gaussian Gram matrix: psd
    assert np.linalg.eigvalsh(K).min() > -1e-10
    rp, ci, w = _dense_csr(K)
    modes = inputs.kmeanspp(X, 3, seed=11)
    A = oracle.unary(X, modes, 1.0)
    lam = 2.0
    Z = softmax(A, axis=1)
    prev = oracle.relaxed(A, Z, rp, ci, w, lam / 2)
    for _ in range(30):
        Z, _, _, _ = oracle.bound_iterate(A, rp, ci, w, lam, Z, 1)
        cur = oracle.relaxed(A, Z, rp, ci, w, lam / 2)
        assert cur <= prev + 1e-12
        prev = cur


def test_relaxed_descends_on_symmetrised_knn_with_shift():
    """Non-psd sparse K: symmetrise the kNN graph and add the diagonal shift
    delta I of footnote 2 (delta = -lambda_min); descent then holds again."""
    X, _ = inputs.blobs(N=60, D=4, n_blobs=3, seed=12)
    idx, _ = oracle.knn(X, 4)
    N = X.shape[0]
    K = np.zeros((N, N))
    for p in range(N):
        K[p, idx[p]] = 1.0
    K = 0.5 * (K + K.T)
    delta = max(0.0, -np.linalg.eigvalsh(K).min()) + 1e-9
    K = K + delta * np.eye(N)
    rp, ci, w = _dense_csr(K)
    A = oracle.unary(X, inputs.kmeanspp(X, 3, seed=12), 2.0)
    lam = 1.5
    Z = softmax(A, axis=1)
    prev = oracle.relaxed(A, Z, rp, ci, w, lam / 2)
    for _ in range(25):
        Z, _, _, _ = oracle.bound_iterate(A, rp, ci, w, lam, Z, 1)
        cur = oracle.relaxed(A, Z, rp, ci, w, lam / 2)
        assert cur <= prev + 1e-12
        prev = cur


# --------------------------------------------------------------------------- modes, labels

def test_mode_update_is_column_argmax_of_softmax():
    g = inputs.rng(13)
    S = g.normal(size=(500, 7)) * 2
    S[300] = S[120]                       # an exact duplicate row: tie -> smaller index
    m, key = oracle.mode_update(S)
    Z = softmax(S, axis=1)
    np.testing.assert_array_equal(m, np.argmax(Z, axis=0))
    np.testing.assert_allclose(key, np.log(Z.max(0)), rtol=1e-12, atol=1e-15)
    col = int(np.argmax(Z[120]))
    S2 = S.copy()
    S2[:, col] = -50.0
    S2[120, col] = S2[300, col] = 50.0
    m2, _ = oracle.mode_update(S2)
    assert m2[col] == 120


def test_log_z_keeps_precision_when_saturated():
    """log z_max = -log(1 + sum_{j != max} e^{s_j - s_max}): with gaps of 60 the
    closed form is -2 e^{-60} (1 - e^{-60}) + ..., which a plain log(softmax)
    rounds to exactly 0."""
    S = np.array([[60.0, 0.0, 0.0], [61.0, 0.0, 0.0]])
    lz = oracle.log_z(S)
    assert lz[0, 0] == pytest.approx(-2 * math.exp(-60), rel=1e-12)
    assert lz[1, 0] == pytest.approx(-2 * math.exp(-61), rel=1e-12)
    m, _ = oracle.mode_update(S)
    assert m[0] == 1                      # the more confident point wins
    np.testing.assert_allclose(lz[:, 1:], log_softmax(S, axis=1)[:, 1:], rtol=1e-13)


def test_labels_argmax_with_ties():
    S = np.array([[0.1, 0.3, 0.3], [2.0, 1.0, 2.0], [0.0, 0.0, 0.0], [-1.0, 5.0, 4.0]])
    np.testing.assert_array_equal(oracle.labels(S), [1, 0, 0, 1])


# --------------------------------------------------------------------------- energy (Eq. 1, Eq. 3)

def _onehot(lab, L):
    Z = np.zeros((len(lab), L))
    Z[np.arange(len(lab)), lab] = 1.0
    return Z


def test_energy_pairwise_is_laplacian_trace():
    """Eq. 3: for symmetric K, (lambda/2) sum k_pq ||z_p - z_q||^2 =
    lambda tr(Z^t (Dg - K) Z) = lambda (sum d_p - sum k_pq z_p^t z_q) at binary Z."""
    X, _ = inputs.blobs(N=80, D=3, n_blobs=4, seed=14)
    N, L = X.shape[0], 4
    idx, _ = oracle.knn(X, 5)
    K = np.zeros((N, N))
    for p in range(N):
        K[p, idx[p]] = 1.0
    K = 0.5 * (K + K.T)
    rp, ci, w = _dense_csr(K)
    lab = inputs.rng(15).integers(0, L, size=N).astype(np.int32)
    modes = np.array([0, 1, 2, 3], np.int32)
    sig, lam = 1.3, 0.7
    E = oracle.energy(X, lab, rp, ci, w, L, modes, sig, lam)
    E_unary_only = oracle.energy(X, lab, rp, ci, w, L, modes, sig, 0.0)
    Z = _onehot(lab, L)
    Lap = np.diag(K.sum(1)) - K
    trace = np.trace(Z.T @ Lap @ Z)
    assert E - E_unary_only == pytest.approx(lam * trace, rel=1e-12)
    assert trace == pytest.approx(K.sum() - np.sum(K * (Z @ Z.T)), rel=1e-12)


def test_energy_unary_closed_form():
    X = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 0.0]], np.float32)
    rp = np.array([0, 1, 2, 3])
    ci = np.array([2, 2, 0])
    lab = np.array([0, 1, 0], np.int32)
    # modes: cluster 0 -> x_0, cluster 1 -> x_1; sigma = 1
    E = oracle.energy(X, lab, rp, ci, None, 2, [0, 1], 1.0, 2.0)
    # unary: k(x0,x0) + k(x1,x1) + k(x2,x0) = 1 + 1 + e^{-1/2}
    # pairwise: edges (0,2) same label, (1,2) different, (2,0) same -> lambda/2 * 2 * 1
    assert E == pytest.approx(-(2 + math.exp(-0.5)) + 2.0, rel=1e-15)


def test_energy_equals_relaxed_at_vertices():
    """Section 2: at simplex vertices the relaxation equals the discrete
    objective up to the constant lambda sum_p d_p (entropy vanishes and
    ||z_p - z_q||^2 = 2 - 2 z_p^t z_q)."""
    X, _ = inputs.blobs(N=70, D=5, n_blobs=3, seed=16)
    rp, ci, w = inputs.random_graph(70, 4, seed=17, weighted=True)
    w = w.astype(np.float64)
    modes = np.array([3, 30, 60], np.int32)
    sig, lam = 2.2, 1.3
    A = oracle.unary(X, modes, sig)
    lab = inputs.rng(18).integers(0, 3, size=70).astype(np.int32)
    E = oracle.energy(X, lab, rp, ci, w, 3, modes, sig, lam)
    R = oracle.relaxed(A, _onehot(lab, 3), rp, ci, w, lam)
    dsum = w.sum()
    assert E == pytest.approx(R + lam * dsum, rel=1e-12)


def test_slk_energy_vs_enumeration_on_separated_blobs():
    """Brute force over all L^N labelings with the modes fixed: the SLK result
    is never below the enumerated minimum and, on well-separated blobs,
    reaches it."""
    g = inputs.rng(19)
    centres = np.array([[0.0, 0.0], [30.0, 0.0]])
    y = np.array([0, 0, 0, 0, 1, 1, 1, 1])
    X = (centres[y] + g.normal(0, 0.5, size=(8, 2))).astype(np.float32)
    k, L, lam = 2, 2, 1.0
    rp, ci, w, d2 = oracle.knn_graph(X, k)
    sig = oracle.sigma(d2)
    res = oracle.solve_graph(X, L, rp, ci, w, sig, lam, np.array([0, 4], np.int32))
    best = min(oracle.energy(X, np.array(lab, np.int32), rp, ci, w, L, res["modes"], sig, lam)
               for lab in itertools.product(range(L), repeat=8))
    assert res["E"] >= best - 1e-12
    assert res["E"] == pytest.approx(best, rel=1e-12)
    assert len(set(zip(y.tolist(), res["labels"].tolist()))) == 2


# --------------------------------------------------------------------------- whole Algorithm 1

def test_solve_recovers_blobs():
    X, y = inputs.blobs(N=600, D=8, n_blobs=4, seed=20)
    m0 = inputs.kmeanspp(X, 4, seed=20)
    out = oracle.solve(X, 4, 5, 1.0, m0)
    assert out["converged"]
    pairs = set(zip(y.tolist(), out["labels"].tolist()))
    assert len(pairs) == 4                 # labels = blob ids up to permutation
    assert len(set(out["modes"].tolist())) == 4
    assert all(0 <= m < 600 for m in out["modes"])
    np.testing.assert_allclose(out["Z"].sum(1), 1.0, atol=1e-14)


def test_golden_worked_example():
    """Hand-worked 4-point example (tests/golden/line4.json): discrete values
    are stored, floating ones are the closed forms written in the fixture."""
    with open(os.path.join(GOLDEN, "line4.json")) as f:
        gold = json.load(f)
    X = np.array(gold["X"], np.float32)
    idx, d2 = oracle.knn(X, gold["k"])
    np.testing.assert_array_equal(idx, gold["knn_idx"])
    sig = oracle.sigma(d2)
    assert sig == gold["sigma"]
    A = oracle.unary(X, gold["init_modes"], sig)
    e = math.exp
    A_want = np.array([[1, e(-50)], [e(-0.5), e(-40.5)], [e(-50), 1], [e(-60.5), e(-0.5)]])
    np.testing.assert_allclose(A, A_want, rtol=1e-14)
    rp = np.arange(5) * gold["k"]
    Z1, _, _, _ = oracle.bound_iterate(A, rp, idx.reshape(-1), None, gold["lambda"],
                                       softmax(A, axis=1), 1)
    Dl = A_want[:, 0] - A_want[:, 1]
    nb = [1, 0, 3, 2]
    logistic = lambda t: 1.0 / (1.0 + math.exp(-t))
    z1_want = [logistic(Dl[p] + math.tanh(Dl[nb[p]] / 2)) for p in range(4)]
    np.testing.assert_allclose(Z1[:, 0], z1_want, rtol=1e-13)
    res = oracle.solve_graph(X, 2, rp, idx.reshape(-1), None, sig, gold["lambda"],
                             np.array(gold["init_modes"], np.int32))
    np.testing.assert_array_equal(res["labels"], gold["labels"])
    np.testing.assert_array_equal(res["modes"], gold["modes"])
    assert res["E"] == pytest.approx(-2 - 2 * math.exp(-0.5), rel=1e-14)


# --------------------------------------------------------------------------- symmetric affinity

def _scipy_sym(rp, ci, w, N):
    import scipy.sparse as sp
    data = np.ones(len(ci)) if w is None else np.asarray(w, np.float64)
    K = sp.csr_matrix((data, ci, rp), shape=(N, N))
    return (0.5 * (K + K.T)).tocsr()


@pytest.mark.parametrize("N,k,weighted", [(50, 4, False), (300, 7, True), (2, 1, False), (1000, 10, True)])
def test_symmetrize_equals_scipy(N, k, weighted):
    """(K + K^t) / 2 (Prop. 1's symmetric affinity) against scipy.sparse:
    same pattern by increasing column (entries that cancel to 0 cannot occur
    with positive weights), same values; mutual edges merge."""
    rp, ci, w = inputs.random_graph(N, k, seed=N + k, weighted=weighted)
    srp, sci, sw = oracle.symmetrize(rp, ci, w, N)
    S = _scipy_sym(rp, ci, w, N)
    S.sort_indices()
    np.testing.assert_array_equal(srp, S.indptr)
    np.testing.assert_array_equal(sci, S.indices)
    np.testing.assert_allclose(sw, S.data, rtol=0, atol=1e-15)
    # symmetric: K'_pq = K'_qp
    D = S.toarray()
    np.testing.assert_array_equal(D, D.T)


def test_symmetrize_mutual_and_one_way_edges_by_hand():
    # 0 -> 1, 1 -> 0 (mutual), 0 -> 2 (one way), binary
    rp = np.array([0, 2, 3, 3], np.int64)
    ci = np.array([1, 2, 0], np.int32)
    srp, sci, sw = oracle.symmetrize(rp, ci, None, 3)
    assert list(srp) == [0, 2, 3, 4]
    assert list(sci) == [1, 2, 0, 0]
    assert list(sw) == [1.0, 0.5, 1.0, 0.5]


def test_solve_on_symmetric_affinity_descends():
    """Prop. 1 with the symmetrised kNN affinity plus the diagonal shift of
    footnote 2: the relaxed objective (lambda/2 on the pairwise term) never
    increases along the oracle's z-updates on oracle.symmetrize's graph."""
    X, _ = inputs.blobs(N=80, D=4, n_blobs=3, seed=21)
    idx, _ = oracle.knn(X, 5)
    N = X.shape[0]
    rp = np.arange(N + 1, dtype=np.int64) * 5
    srp, sci, sw = oracle.symmetrize(rp, idx.reshape(-1), None, N)
    K = np.zeros((N, N))
    for p in range(N):
        K[p, sci[srp[p]:srp[p + 1]]] = sw[srp[p]:srp[p + 1]]
    delta = max(0.0, -np.linalg.eigvalsh(K).min()) + 1e-9
    rp2, ci2, w2 = _dense_csr(K + delta * np.eye(N))
    A = oracle.unary(X, inputs.kmeanspp(X, 3, seed=21), 2.0)
    lam = 1.5
    Z = softmax(A, axis=1)
    prev = oracle.relaxed(A, Z, rp2, ci2, w2, lam / 2)
    for _ in range(25):
        Z, _, _, _ = oracle.bound_iterate(A, rp2, ci2, w2, lam, Z, 1)
        cur = oracle.relaxed(A, Z, rp2, ci2, w2, lam / 2)
        assert cur <= prev + 1e-12
        prev = cur
