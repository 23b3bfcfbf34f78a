"""GPU parity of SLK-MS (modes via mean-shift) through the C-ABI against the
FP64 oracle on the same seeded inputs.

Mode vectors are compared within M_TOL * sigma (max-abs).  The float32
kernel differs from the float64 oracle in each weight exponent
s = log z - ||x - m||^2 / (2 sigma^2) by about (eps32 * D) * d2 / (2 sigma^2)
plus a few ulp of log z (eps32 = 2^-24, up to ~5e-6 at D = 784 for the
points that carry weight); a relative weight error e moves a weighted mean
by at most e times the weighted spread of the points (a few sigma), and
the contraction of the fixed-point iteration keeps later iterations from
adding up beyond that: 2e-4 sigma covers this with margin.  Labels must be
identical (near-ties of the logits bounded as in the SLK-BO tests), Z within
1e-5, E within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M_TOL = 2e-4     # x sigma
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


def _case(N, D, L, seed):
    """Blobs with L centres, starting modes near K-means++ seeds, sigma of
    the within-blob distance scale, and peaked unary logits A."""
    X, _ = inputs.blobs(N=N, D=D, n_blobs=max(L, 1), centre_var=25.0, seed=seed)
    g = inputs.rng(seed + 1)
    m0 = inputs.kmeanspp(X, L, seed=seed)
    M0 = (X[m0].astype(np.float64) + 0.3 * g.normal(size=(L, D))).astype(np.float32)
    sig = float(0.5 * np.sqrt(2.0 * D))
    A = (6.0 * oracle.unary_vec(X, M0.astype(np.float64), sig)).astype(np.float32)
    return X, M0, sig, A


MS_CASES = [
    (2000, 16, 5, 1810),    # the 2000 x 16 blobs shape
    (3000, 784, 10, 2),     # the 70000 x 784, L=10 kernel shape (16 rows, 12 labels, 4 features/thread)
    (3000, 3, 4, 3),        # D % 4 != 0: plain loads instead of bulk copies
    (1500, 300, 13, 4),     # 2 features per thread, 16-label group
    (800, 1500, 8, 5),      # 8-row tiles, 8 features per thread
    (300, 3000, 6, 6),      # 4-row tiles, 16 features per thread, two label groups
    (500, 64, 40, 7),       # three label groups
    (37, 7, 3, 8),          # ragged last tile
    (2, 5, 1, 9),           # two points, one mode
    (1000, 128, 100, 10),   # the 1e6 x 128, L=100 kernel shape
]


@pytest.mark.parametrize("N,D,L,seed", MS_CASES)
def test_mean_shift_fixed_iterations(slk, N, D, L, seed):
    X, M0, sig, A = _case(N, D, L, seed)
    logZ = oracle.log_z(A.astype(np.float64))
    for iters in (1, 3, 10):
        M = dev(M0)
        it, sh, labels = slk.mean_shift(dev(X), dev(A), None, None, None, None, 1.0, sig, M, iters,
                                        tol=-1.0)
        Mo, ito, sho = oracle.mean_shift(X, logZ, M0.astype(np.float64), sig, iters, -1.0)
        assert it == ito == iters
        err = np.abs(host(M).astype(np.float64) - Mo).max()
        print(f"mean-shift N={N} D={D} L={L} iters={iters}: max|dM|/sigma = {err / sig:.3e}")
        assert err <= M_TOL * sig, (iters, err / sig)
        assert sh == pytest.approx(sho, rel=1e-2, abs=M_TOL * sig)
        ol = oracle.labels(A.astype(np.float64))
        gl = host(labels)
        for p in np.nonzero(gl != ol)[0]:
            assert abs(A[p, gl[p]] - A[p, ol[p]]) <= KEY_TIE


@pytest.mark.parametrize("N,D,L,seed", [(2000, 16, 5, 1810), (3000, 784, 10, 2), (500, 64, 40, 7)])
def test_mean_shift_until_converged(slk, N, D, L, seed):
    X, M0, sig, A = _case(N, D, L, seed)
    logZ = oracle.log_z(A.astype(np.float64))
    tol = 1e-5
    M = dev(M0)
    it, sh, _ = slk.mean_shift(dev(X), dev(A), None, None, None, None, 1.0, sig, M, 200, tol=tol)
    Mo, ito, sho = oracle.mean_shift(X, logZ, M0.astype(np.float64), sig, 200, tol)
    assert it < 200 and sh <= tol * sig
    assert abs(it - ito) <= 1
    assert np.abs(host(M).astype(np.float64) - Mo).max() <= M_TOL * sig


@pytest.mark.parametrize("weighted", [False, True])
def test_mean_shift_weights_from_last_update(slk, weighted):
    """z enters through the logits of the last z-update (A + lambda K Z_prev)."""
    N, D, L, k = 1200, 24, 6, 5
    X, M0, sig, A = _case(N, D, L, 11)
    rp, ci, w = inputs.random_graph(N, k, seed=12, weighted=weighted)
    Zp = inputs.random_simplex_rows(N, L, seed=13)
    lam = 1.5
    M = dev(M0)
    it, _, labels = slk.mean_shift(dev(X), dev(A), dev(Zp), dev(rp), dev(ci),
                                   None if w is None else dev(w), lam, sig, M, 5)
    S = oracle.logits(A, rp, ci, w, lam, Zp)
    Mo, _, _ = oracle.mean_shift(X, oracle.log_z(S), M0.astype(np.float64), sig, 5)
    assert it == 5
    assert np.abs(host(M).astype(np.float64) - Mo).max() <= M_TOL * sig
    ol = oracle.labels(S)
    gl = host(labels)
    for p in np.nonzero(gl != ol)[0]:
        assert abs(S[p, gl[p]] - S[p, ol[p]]) <= KEY_TIE


def test_mean_shift_saturated_and_far_modes(slk):
    """Logit gaps of 60 (float32 z is 0 or 1) and a mode far from every
    point: the log-domain weights keep both finite and ordered."""
    N, D, L = 256, 8, 3
    g = inputs.rng(21)
    X = g.normal(size=(N, D)).astype(np.float32)
    A = np.zeros((N, L), np.float32)
    A[:, 0] = 60.0 * (np.arange(N) % 2)
    A[:, 1] = 30.0
    M0 = np.zeros((L, D), np.float32)
    M0[2, 0] = 400.0                      # exp(-400^2 / 2) underflows in float64 too
    sig = 1.0
    M = dev(M0)
    slk.mean_shift(dev(X), dev(A), None, None, None, None, 1.0, sig, M, 4)
    Mo, _, _ = oracle.mean_shift(X, oracle.log_z(A.astype(np.float64)), M0.astype(np.float64),
                                 sig, 4)
    Mg = host(M).astype(np.float64)
    assert np.all(np.isfinite(Mg))
    assert np.abs(Mg - Mo).max() <= M_TOL * sig


def test_mean_shift_full_size_two_iterations(slk):
    """The 70000 x 784, L=10 shape the SLK-MS benchmark times, two
    iterations from K-means++ seeds, against the oracle."""
    X, _ = inputs.mnist_like()
    L = 10
    m0 = inputs.kmeanspp(X, L, seed=1810)
    M0 = X[m0].astype(np.float64)
    sig = 3.0
    A64 = 6.0 * oracle.unary_vec(X, M0, sig)
    A = A64.astype(np.float32)
    M = dev(M0.astype(np.float32))
    it, _, _ = slk.mean_shift(dev(X), dev(A), None, None, None, None, 1.0, sig, M, 2)
    Mo, _, _ = oracle.mean_shift(X, oracle.log_z(A.astype(np.float64)), M0, sig, 2)
    assert it == 2
    assert np.abs(host(M).astype(np.float64) - Mo).max() <= M_TOL * sig


@pytest.mark.parametrize("N,D,L", [(2000, 16, 5), (333, 31, 33), (500, 784, 10)])
def test_unary_vec_matches_oracle(slk, N, D, L):
    X, M0, sig, _ = _case(N, D, L, 31)
    A, Z0 = slk.unary_vec(dev(X), dev(M0), sig)
    Ao = oracle.unary_vec(X, M0.astype(np.float64), sig)
    assert np.abs(host(A) - Ao).max() <= 1e-6
    assert np.abs(host(Z0) - oracle.softmax_rows(Ao)).max() <= 1e-6


@pytest.mark.parametrize("weighted", [False, True])
def test_energy_vec_matches_oracle(slk, weighted):
    N, D, L, k = 1500, 20, 7, 5
    X, M0, sig, _ = _case(N, D, L, 41)
    rp, ci, w = inputs.random_graph(N, k, seed=42, weighted=weighted)
    lab = inputs.rng(43).integers(0, L, N).astype(np.int32)
    E = slk.energy_vec(dev(X), dev(lab), dev(rp), dev(ci), None if w is None else dev(w), dev(M0),
                       sig, 1.3)
    Eo = oracle.energy_vec(X, lab, rp, ci, w, M0.astype(np.float64), sig, 1.3)
    assert E == pytest.approx(Eo, rel=E_RTOL)


def _compare_solve_ms(out, ref, sig, strict=True, z_tol=Z_TOL):
    """strict: fixed mean-shift counts on both sides (tol_ms < 0), so only
    rounding separates them.  Otherwise each side stops its mean-shift at
    tol_ms * sigma and the two can stop one iteration apart: the modes may
    then differ by up to about tol_ms * sigma / (1 - r) (r < 0.9, the
    contraction of the iteration), 1e-4 sigma, which moves a, and through
    it Z, by up to ~1e-4 as well; labels must still agree."""
    Z, labels, M, st = out
    assert st["outer_iters"] == ref["outer"]
    assert st["converged"] == int(ref["converged"])
    np.testing.assert_array_equal(host(labels), ref["labels"])
    if strict:
        assert st["ms_iters_total"] == ref["ms_total"]
        m_err = np.abs(host(M).astype(np.float64) - ref["M"]).max()
        z_err = np.abs(host(Z) - ref["Z"]).max()
        print(f"solve_ms: max|dM|/sigma = {m_err / sig:.3e}, max|dZ| = {z_err:.3e}")
        assert m_err <= M_TOL * sig
        assert z_err <= z_tol
        assert st["energy"] == pytest.approx(ref["E"], rel=E_RTOL)
    else:
        assert abs(st["ms_iters_total"] - ref["ms_total"]) <= st["outer_iters"]
        assert np.abs(host(M).astype(np.float64) - ref["M"]).max() <= 1e-3 * sig
        assert np.abs(host(Z) - ref["Z"]).max() <= 1e-3
        assert st["energy"] == pytest.approx(ref["E"], rel=1e-5)


@pytest.mark.parametrize("strict", [True, False])
def test_solve_ms_blobs_matches_oracle(slk, strict):
    """2000 x 16 blobs, L=5, k=5, lambda=1, sigma = median kNN distance."""
    X, _ = inputs.blobs()
    L, k, lam = 5, 5, 1.0
    m0 = inputs.kmeanspp(X, L, seed=1810)
    tol_ms = -1.0 if strict else 1e-5
    ref = oracle.solve_ms(X, L, k, lam, m0, max_ms=25, tol_ms=tol_ms)
    p = slk.default_params(max_ms=25, tol_ms=tol_ms)
    out = slk.solve_ms(dev(X), L, k, lam, dev(m0), sigma=ref["sigma"], params=p)
    _compare_solve_ms(out, ref, ref["sigma"], strict)
    assert ref["converged"]


@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("seed", [3, 4])
def test_solve_ms_multi_outer_matches_oracle(slk, seed, strict):
    """Overlapping blobs and a bad seed so that the modes move over several
    outer iterations.  Unlike SLK-BO, whose modes are exact data points, the
    mean-shift modes carry the float32 arithmetic of the mean (~1e-7 sigma,
    tested above), which moves a by ~1e-7 (|x - m| / sigma) and reaches Z
    through the inner fixed point z = softmax(a + lambda K z); with lambda = 2,
    k = 5 and overlapping blobs that map amplifies a change of a by up to
    (1 - lambda |J K|)^-1 ~ 30-100 (J the soft-max Jacobian), so Z is held to
    5e-5 here and to 1e-5 on the separated blobs above."""
    X, _ = inputs.blobs(N=1500, D=4, n_blobs=6, centre_var=6.0, seed=seed)
    L, k, lam = 6, 5, 2.0
    m0 = np.arange(L, dtype=np.int32)
    tol_ms = -1.0 if strict else 1e-5
    ref = oracle.solve_ms(X, L, k, lam, m0, max_outer=8, max_ms=25, tol_ms=tol_ms)
    p = slk.default_params(max_outer=8, max_ms=25, tol_ms=tol_ms)
    out = slk.solve_ms(dev(X), L, k, lam, dev(m0), sigma=ref["sigma"], params=p)
    assert ref["outer"] >= 2
    _compare_solve_ms(out, ref, ref["sigma"], strict, z_tol=5e-5)


def test_solve_ms_mnist_like_full_size(slk):
    """The SLK-MS benchmark configuration (70000 x 784, L=10, k=5, bf16 kNN
    tiles): properties that hold at any size."""
    X, _ = inputs.mnist_like()
    L, k, lam = 10, 5, 1.0
    m0 = inputs.kmeanspp(X, L, seed=1810)
    Xd = dev(X)
    p = slk.default_params(knn_precision="bf16_rerank")
    Z, labels, M, st = slk.solve_ms(Xd, L, k, lam, dev(m0), params=p)
    assert st["converged"] == 1 and st["ms_iters_total"] >= st["outer_iters"]
    Zh = host(Z).astype(np.float64)
    np.testing.assert_allclose(Zh.sum(1), 1.0, atol=1e-5)
    Mh = host(M).astype(np.float64)
    assert np.all(np.isfinite(Mh))
    # mean-shift modes are weighted means: inside the bounding box of the data
    assert np.all(Mh >= X.min(0) - 1e-6) and np.all(Mh <= X.max(0) + 1e-6)
    lab = host(labels)
    srt = np.sort(Zh, 1)
    clear = srt[:, -1] - srt[:, -2] > 1e-6
    np.testing.assert_array_equal(lab[clear], np.argmax(Zh, 1)[clear])
    # the energy is Eq. (1) on the returned labels and modes (the solve evaluates
    # it with the float64 mode state, the check with the float32 modes it returns)
    g = slk.knn_graph(Xd, k, precision="bf16_rerank")
    E = slk.energy_vec(Xd, labels, g.row_ptr, g.col_idx, None, M, st["sigma"], lam)
    assert E == pytest.approx(st["energy"], rel=1e-9)
    d2 = ((X.astype(np.float64) - Mh[lab]) ** 2).sum(1)
    col = host(g.col_idx).reshape(-1, k)
    cut = (lab[col] != lab[:, None]).sum()
    E64 = -np.exp(-d2 / (2.0 * st["sigma"] ** 2)).sum() + lam * cut
    assert E64 == pytest.approx(st["energy"], rel=1e-9)
    # one more mean-shift pass from the final modes with the final z moves them little
    # (the outer loop stopped because they moved <= tol_modes * sigma)
    assert st["outer_iters"] <= 50


def test_mean_shift_invalid_arguments(slk):
    X = dev(np.zeros((10, 4), np.float32))
    A = dev(np.zeros((10, 2), np.float32))
    M = dev(np.zeros((2, 4), np.float32))
    with pytest.raises(slk.SlkError):
        slk.mean_shift(X, A, None, None, None, None, 1.0, 0.0, M, 3)       # sigma <= 0
    with pytest.raises(slk.SlkError):
        slk.mean_shift(X, A, None, None, None, None, 1.0, 1.0, M, -1)      # max_iters < 0
    Xw = dev(np.zeros((10, 5000), np.float32))
    Mw = dev(np.zeros((2, 5000), np.float32))
    with pytest.raises(slk.SlkError):
        slk.mean_shift(Xw, A, None, None, None, None, 1.0, 1.0, Mw, 3)     # D > SLK_MS_MAX_D
