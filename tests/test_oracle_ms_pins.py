"""Pins of the SLK-MS part of the FP64 oracle (modes via mean-shift).

Each test checks the oracle against something other than its own formula:
closed forms of the Gaussian kernel density, the stationarity and ascent
properties of Gaussian mean-shift (the update is a fixed-point iteration on
the weighted kernel density f_l(m) = sum_p z_{p,l} k(x_p, m), whose fixed
points are the stationary points of f_l and along which f_l never decreases),
special cases that reduce to already pinned SLK-BO functions, and blob
recovery.
"""
import numpy as np
import pytest

import oracle

scipy_opt = pytest.importorskip("scipy.optimize")


def kde(X, z, m, sig):
    """Weighted kernel density f(m) = sum_p z_p exp(-||x_p - m||^2 / (2 sig^2))."""
    d2 = ((np.asarray(X, np.float64) - m) ** 2).sum(1)
    return float((z * np.exp(-d2 / (2 * sig * sig))).sum())


def kde_grad_fd(X, z, m, sig, h=1e-5):
    g = np.zeros_like(m)
    for j in range(m.size):
        e = np.zeros_like(m)
        e[j] = h
        g[j] = (kde(X, z, m + e, sig) - kde(X, z, m - e, sig)) / (2 * h)
    return g


def test_unary_vec_equals_point_modes():
    g = np.random.default_rng(3)
    X = g.normal(size=(40, 7)).astype(np.float32)
    modes = np.array([4, 11, 39], np.int32)
    A_pts = oracle.unary(X, modes, 1.7)
    A_vec = oracle.unary_vec(X, X[modes].astype(np.float64), 1.7)
    np.testing.assert_array_equal(A_vec, A_pts)


def test_unary_vec_closed_form():
    X = np.array([[1.5, 0.0], [0.5, 2.0]], np.float32)
    M = np.array([[0.5, 0.0], [0.5, 2.0]])
    A = oracle.unary_vec(X, M, 2.0)
    np.testing.assert_allclose(A, [[np.exp(-1 / 8), np.exp(-(1 + 4) / 8)],
                                   [np.exp(-4 / 8), 1.0]], rtol=1e-15)


@pytest.mark.parametrize("a,sig", [(0.5, 1.0), (0.8, 1.3)])
def test_two_points_unimodal_converges_to_midpoint(a, sig):
    # Two equal Gaussians at -a, +a: the density is unimodal for a < sig, mode 0.
    X = np.array([[-a], [a]], np.float32)
    lz = np.log(np.full((2, 1), 0.5))
    M, it, sh = oracle.mean_shift(X, lz, [[0.9 * a]], sig, 500, 1e-13)
    assert it < 500
    assert abs(M[0, 0]) < 1e-10


@pytest.mark.parametrize("a,sig,z1", [(2.0, 1.0, 0.5), (1.5, 1.0, 0.5), (2.0, 1.0, 0.8),
                                      (3.0, 2.0, 0.3)])
def test_two_points_bimodal_root(a, sig, z1):
    # Stationary points of z1 k(m - a) + z2 k(m + a): zeros of the derivative
    # -z1 (m - a) k(m - a) - z2 (m + a) k(m + a) (sigma^2 dropped), solved by a
    # bracketing root finder on the right-hand mode.
    a32 = float(np.float32(a))
    z2 = 1.0 - z1

    def fprime(m):
        k1 = np.exp(-(m - a32) ** 2 / (2 * sig * sig))
        k2 = np.exp(-(m + a32) ** 2 / (2 * sig * sig))
        return -z1 * (m - a32) * k1 - z2 * (m + a32) * k2

    lo = 0.5 * a32 if (z1 >= z2 or a32 > 1.4 * sig) else a32 * 0.9
    root = scipy_opt.brentq(fprime, lo, a32 + 3 * sig, xtol=1e-15)
    X = np.array([[a], [-a]], np.float32)
    lz = np.log(np.array([[z1], [z2]]))
    M, it, _ = oracle.mean_shift(X, lz, [[a32]], sig, 2000, 1e-14)
    assert abs(M[0, 0] - root) < 1e-10


def test_stationary_and_local_max_per_label():
    # L = 2 labels with different weights over the same points, D = 3 != L.
    g = np.random.default_rng(11)
    X = np.concatenate([g.normal(0, 1, (25, 3)), g.normal(4, 1, (25, 3))]).astype(np.float32)
    z = g.dirichlet([0.7, 0.7], size=50)
    sig = 1.2
    M0 = X[[3, 30]].astype(np.float64)
    M, it, sh = oracle.mean_shift(X, np.log(z), M0, sig, 5000, 1e-12)
    assert it < 5000
    for l in range(2):
        grad = kde_grad_fd(X, z[:, l], M[l], sig)
        scale = kde(X, z[:, l], M[l], sig) / sig
        assert np.abs(grad).max() < 1e-7 * scale
        f0 = kde(X, z[:, l], M[l], sig)
        for _ in range(20):
            d = g.normal(size=3)
            d *= 1e-3 / np.linalg.norm(d)
            assert kde(X, z[:, l], M[l] + d, sig) <= f0


def test_density_never_decreases():
    g = np.random.default_rng(5)
    X = g.normal(size=(60, 4)).astype(np.float32) * 2.0
    z = g.dirichlet([1.0, 1.0, 1.0], size=60)
    sig = 0.9
    M = X[[0, 1, 2]].astype(np.float64)
    f_prev = [kde(X, z[:, l], M[l], sig) for l in range(3)]
    for _ in range(30):
        M, it, _ = oracle.mean_shift(X, np.log(z), M, sig, 1)
        assert it == 1
        f = [kde(X, z[:, l], M[l], sig) for l in range(3)]
        for l in range(3):
            assert f[l] >= f_prev[l] * (1 - 1e-14)
        f_prev = f


def test_single_weighted_point():
    # A weight that is zero for every point but one: the mode is that point.
    X = np.array([[0.0, 1.0], [3.0, -2.0], [5.0, 5.0]], np.float32)
    lz = np.array([[-np.inf], [0.0], [-np.inf]])
    M, it, _ = oracle.mean_shift(X, lz, [[4.0, 4.0]], 1.0, 1)
    np.testing.assert_array_equal(M[0], [3.0, -2.0])
    # started at its fixed point, the first iteration already meets the tolerance
    M, it, sh = oracle.mean_shift(X, lz, [[3.0, -2.0]], 1.0, 50, 1e-6)
    assert it == 1 and sh == 0.0


def test_weight_scale_and_far_modes():
    # z_{p,l} -> c z_{p,l} leaves the ratio unchanged; a mode far from every
    # point (every kernel value below the smallest double) still gets the
    # mean of the closest points' weights instead of 0/0.
    g = np.random.default_rng(2)
    X = g.normal(size=(30, 2)).astype(np.float32)
    z = g.dirichlet([1.0, 1.0], size=30)
    M0 = np.array([[0.3, 0.1], [-0.2, 0.4]])
    M1, _, _ = oracle.mean_shift(X, np.log(z), M0, 1.0, 3)
    M2, _, _ = oracle.mean_shift(X, np.log(z) - 800.0, M0, 1.0, 3)
    np.testing.assert_allclose(M2, M1, rtol=0, atol=1e-13)
    far = np.array([[100.0, 0.0]])
    Mf, _, _ = oracle.mean_shift(X, np.log(z[:, :1]), far, 1.0, 1)
    assert np.all(np.isfinite(Mf))
    # exp(-(100 - x)^2 / 2) ~ exp(-(100^2 - 200 x) / 2): the point with the largest x dominates
    assert np.linalg.norm(Mf[0] - X[np.argmax(X[:, 0])]) < 1e-6


def test_iteration_count_rule():
    g = np.random.default_rng(9)
    X = (g.normal(size=(40, 2)) * 4.0).astype(np.float32)
    z = g.dirichlet([1.0, 1.0], size=40)
    sig, tol = 3.2, 1e-3            # sigma far from 1: the rule is relative to sigma
    M0 = X[[0, 1]].astype(np.float64)
    _, it_fixed, _ = oracle.mean_shift(X, np.log(z), M0, sig, 7, -1.0)
    assert it_fixed == 7
    M = M0.copy()
    expect = None
    for t in range(1, 200):
        Mn, _, _ = oracle.mean_shift(X, np.log(z), M, sig, 1)
        shift = np.linalg.norm(Mn - M, axis=1).max()
        M = Mn
        if shift <= tol * sig:
            expect = t
            break
    assert expect is not None
    Mt, it, sh = oracle.mean_shift(X, np.log(z), M0, sig, 200, tol)
    assert it == expect
    np.testing.assert_allclose(Mt, M, rtol=0, atol=1e-14)
    assert sh <= tol * sig


def test_energy_vec_equals_point_modes():
    g = np.random.default_rng(4)
    X = g.normal(size=(50, 3)).astype(np.float32)
    rp, ci, w, d2 = oracle.knn_graph(X, 4)
    lab = g.integers(0, 3, 50).astype(np.int32)
    modes = np.array([7, 20, 41], np.int32)
    for ww in (None, oracle.heat_weights(d2, 1.1)):
        E1 = oracle.energy(X, lab, rp, ci, ww, 3, modes, 1.1, 1.5)
        E2 = oracle.energy_vec(X, lab, rp, ci, ww, X[modes].astype(np.float64), 1.1, 1.5)
        assert E2 == pytest.approx(E1, rel=1e-15, abs=0)


def test_energy_vec_closed_form():
    # 3 points on a line, modes off the data: -sum k(x_p, m_{l_p}) + lambda/2 * cut.
    X = np.array([[0.0], [1.0], [3.0]], np.float32)
    rp = np.array([0, 1, 2, 3], np.int64)
    ci = np.array([1, 0, 1], np.int32)           # 0->1, 1->0, 2->1
    lab = np.array([0, 0, 1], np.int32)
    M = np.array([[0.5], [2.5]])
    E = oracle.energy_vec(X, lab, rp, ci, None, M, 1.0, 2.0)
    un = 2 * np.exp(-0.25 / 2) + np.exp(-0.25 / 2)
    assert E == pytest.approx(-un + 0.5 * 2.0 * 2.0, rel=1e-14)


def _one_outer_by_parts(X, L, rp, ci, w, sig, lam, M0, max_inner, tol, max_ms, tol_ms):
    A = oracle.unary_vec(X, M0, sig)
    Z0 = oracle.softmax_rows(A)
    Z, Zp, it, _ = oracle.bound_iterate(A, rp, ci, w, lam, Z0, max_inner, tol)
    S = oracle.logits(A, rp, ci, w, lam, Zp) if it > 0 else A
    M, ms, _ = oracle.mean_shift(X, oracle.log_z(S), M0, sig, max_ms, tol_ms)
    lab = oracle.labels(S)
    E = oracle.energy_vec(X, lab, rp, ci, w, M, sig, lam)
    return Z, lab, M, E, it, ms


def test_solve_ms_one_outer_is_the_composition():
    from paper_1810_13044_gb300 import inputs
    X, _ = inputs.blobs(300, 5, 3, seed=21)
    rp, ci, w, d2 = oracle.knn_graph(X, 5)
    sig = oracle.sigma(d2)
    M0 = X[[5, 100, 200]].astype(np.float64)
    r = oracle.solve_ms_graph(X, 3, rp, ci, None, sig, 1.0, M0, max_outer=1, max_inner=30,
                              tol=1e-6, max_ms=40, tol_ms=1e-5)
    Z, lab, M, E, it, ms = _one_outer_by_parts(X, 3, rp, ci, None, sig, 1.0, M0, 30, 1e-6, 40, 1e-5)
    np.testing.assert_array_equal(r["Z"], Z)
    np.testing.assert_array_equal(r["labels"], lab)
    np.testing.assert_array_equal(r["M"], M)
    assert r["E"] == E and r["inner_total"] == it and r["ms_total"] == ms and r["outer"] == 1


def test_solve_ms_outer_stopping_rule():
    from paper_1810_13044_gb300 import inputs
    X, _ = inputs.blobs(240, 4, 3, seed=8)
    X = X * np.float32(6.0)         # sigma far from 1: the rule is relative to sigma
    rp, ci, w, d2 = oracle.knn_graph(X, 5)
    sig = oracle.sigma(d2)
    assert sig > 3.0
    init = inputs.kmeanspp(X, 3, seed=8)
    M0 = X[init].astype(np.float64)
    # mode moves of the outer steps, each run from scratch with a fixed count
    prev, moves, Ms = M0, [], []
    for t in range(1, 7):
        r = oracle.solve_ms_graph(X, 3, rp, ci, None, sig, 1.0, M0, max_outer=t, tol_outer=-1.0)
        moves.append(np.linalg.norm(r["M"] - prev, axis=1).max())
        Ms.append(r["M"])
        prev = r["M"]
    # a threshold just above one move: the outer loop stops exactly at that step
    j = next(j for j in range(1, 6) if moves[j] > 0 and min(moves[:j]) > 1.02 * moves[j])
    tol_outer = 1.01 * moves[j] / sig
    full = oracle.solve_ms_graph(X, 3, rp, ci, None, sig, 1.0, M0, max_outer=30,
                                 tol_outer=tol_outer)
    assert full["converged"] and full["outer"] == j + 1
    np.testing.assert_array_equal(full["M"], Ms[j])
    capped = oracle.solve_ms_graph(X, 3, rp, ci, None, sig, 1.0, M0, max_outer=j,
                                   tol_outer=tol_outer)
    assert not capped["converged"] and capped["outer"] == j


def test_solve_ms_recovers_blobs():
    from paper_1810_13044_gb300 import inputs
    X, y = inputs.blobs(2000, 16, 5, seed=1810)
    init = inputs.kmeanspp(X, 5, seed=1810)
    r = oracle.solve_ms(X, 5, 5, 1.0, init)
    assert r["converged"]
    lab = r["labels"]
    # labels agree with the generating blobs up to a permutation
    perm = {}
    for l in range(5):
        vals, cnt = np.unique(y[lab == l], return_counts=True)
        assert cnt.max() == cnt.sum()
        perm[l] = int(vals[np.argmax(cnt)])
    assert len(set(perm.values())) == 5
    # every mode sits near the mean of its blob (the smoothed density of a
    # unit-variance Gaussian blob peaks at its centre)
    for l in range(5):
        centre = X[y == perm[l]].astype(np.float64).mean(0)
        assert np.linalg.norm(r["M"][l] - centre) < 0.5
