"""GPU parity of the starting modes (Section 4.2: nearest-seed assignment,
then the mode definition of Eq. (1)) through the C-ABI against the FP64
oracle.

Integer results are compared exactly except where float rounding decides
them between near-equal candidates:
  assignment: the oracle's float64 squared distances to the two seeds agree
    within 1e-6 relative (the GPU sums float32 squares of float32
    differences in chunks of 32, in float64);
  modes: the oracle's cluster density at the GPU's mode is within DENS_RTOL
    of the oracle's maximum.
DENS_RTOL: the reported densities (and the final choice among the
certified candidates) come from float32 differences whose squares are
summed in float32 chunks of 8 and then in float64: d2 is within ~9u
relative (u = 2^-24), so a kernel value k = exp(-d2 / (2 sigma^2)) within
9u d2 / (2 sigma^2) relative; the terms that carry weight have d2 below
~40 sigma^2, which bounds the relative error of a density by ~1.1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DENS_RTOL = 2e-5


@pytest.fixture(scope="module")
def slk():
    from paper_1810_13044_gb300 import build, slk as _slk
    build.build()
    return _slk


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _check_assign(X, seeds, g_assign, o_assign):
    diff = np.nonzero(g_assign != o_assign)[0]
    for p in diff:
        d = ((X[p].astype(np.float64) - X[seeds[[g_assign[p], o_assign[p]]]].astype(np.float64)) ** 2).sum(1)
        assert abs(d[0] - d[1]) <= 1e-6 * max(d.max(), 1e-30), (p, d)
    assert len(diff) <= max(1, len(g_assign) // 1000)


def _check_modes(X, sig, g_modes, g_dens, o_modes, o_dens, o_assign):
    L = len(o_modes)
    for l in range(L):
        if o_dens[l] == 0.0:                      # empty cluster: keeps its seed
            assert g_dens[l] == 0.0 and g_modes[l] == o_modes[l]
            continue
        if g_modes[l] != o_modes[l]:
            f = oracle.cluster_density(X, o_assign, l, sig, np.array([g_modes[l]]))[0]
            assert f >= o_dens[l] * (1 - DENS_RTOL), (l, g_modes[l], o_modes[l], f, o_dens[l])
        assert g_dens[l] == pytest.approx(o_dens[l], rel=DENS_RTOL)


@pytest.mark.parametrize("N,D,L,seed", [
    (2000, 16, 5, 1810),      # the 2000 x 16 blobs workload
    (3000, 784, 10, 2),       # the 70000 x 784 shape
    (300, 7, 3, 3),           # ragged tiles, D % 16 != 0
    (1500, 64, 40, 4),        # many clusters, uneven sizes
    (129, 130, 1, 5),         # one cluster
    (1, 3, 1, 6),             # one point
])
def test_initial_modes_match_oracle(slk, N, D, L, seed):
    if (N, D) == (2000, 16):
        X, _ = inputs.blobs(seed=seed)
    elif D == 784:
        X, _ = inputs.mnist_like(N=N, seed=seed)
    else:
        X, _ = inputs.blobs(N=N, D=D, n_blobs=max(L, 1), centre_var=9.0, seed=seed)
    seeds = inputs.kmeanspp(X, L, seed=seed) if N > 1 else np.zeros(1, np.int32)
    sig = float(0.4 * np.sqrt(2.0 * D))
    o_modes, o_assign, o_dens = oracle.initial_modes(X, seeds, sig)
    st = {}
    g_modes, g_assign, g_dens = slk.initial_modes(dev(X), dev(seeds), sig, stats=st)
    _check_assign(X, seeds, host(g_assign), o_assign)
    _check_modes(X, sig, host(g_modes), np.array(g_dens), o_modes, o_dens, o_assign)
    print(f"initial modes N={N} D={D} L={L}: {st['candidates']} exact recomputes")
    assert 1 <= st["candidates"] <= N * L


def test_initial_modes_duplicate_and_empty_cluster(slk):
    g = inputs.rng(9)
    X = g.normal(size=(400, 6)).astype(np.float32)
    X[250] = X[17]                                # a duplicate: wins under a narrow kernel
    seeds = np.array([17, 17, 300], np.int32)     # label 1 ties with label 0: empty
    o_modes, o_assign, o_dens = oracle.initial_modes(X, seeds, 1e-3)
    g_modes, g_assign, g_dens = slk.initial_modes(dev(X), dev(seeds), 1e-3)
    np.testing.assert_array_equal(host(g_assign), o_assign)
    np.testing.assert_array_equal(host(g_modes), o_modes)
    assert host(g_modes)[1] == 17 and g_dens[1] == 0.0
    assert g_dens[0] == pytest.approx(2.0, rel=1e-6)


def test_initial_modes_full_size_sampled(slk):
    """The 70000 x 784, L=10 workload: the oracle's assignment in full, then
    the oracle's cluster density at the GPU's mode and at sampled points of
    each cluster (its seed among them)."""
    X, _ = inputs.mnist_like()
    L = 10
    seeds = inputs.kmeanspp(X, L, seed=1810)
    sig = 3.0
    st = {}
    g_modes, g_assign, g_dens = slk.initial_modes(dev(X), dev(seeds), sig, stats=st)
    gm, ga = host(g_modes), host(g_assign)
    print(f"initial modes full size: {st['candidates']} exact recomputes")
    assert st["candidates"] < X.shape[0]        # the bound leaves a small candidate set
    o_assign = np.empty(X.shape[0], np.int32)
    d = np.full(X.shape[0], np.inf)
    X64 = X.astype(np.float64)
    for l, s in enumerate(seeds):
        dl = ((X64 - X64[s]) ** 2).sum(1)
        better = dl < d
        o_assign[better] = l
        d[better] = dl[better]
    _check_assign(X, seeds, ga, o_assign)
    rng = inputs.rng(10)
    for l in range(L):
        members = np.nonzero(o_assign == l)[0]
        sample = np.concatenate([[gm[l], seeds[l]], rng.choice(members, size=min(40, len(members)),
                                                               replace=False)])
        f = oracle.cluster_density(X, o_assign, l, sig, sample)
        assert f[0] >= f.max() * (1 - DENS_RTOL)
        assert g_dens[l] == pytest.approx(f[0], rel=DENS_RTOL)


def test_solve_with_refined_start_matches_oracle(slk):
    """slk_solve with refine_init: Algorithm 1 from the starting modes."""
    X, _ = inputs.blobs()
    L, k, lam = 5, 5, 1.0
    seeds = inputs.kmeanspp(X, L, seed=1810)
    idx, d2 = oracle.knn(X, k)
    sig = oracle.sigma(d2)
    o_start, _, _ = oracle.initial_modes(X, seeds, sig)
    ref = oracle.solve(X, L, k, lam, o_start, sig=sig)
    p = slk.default_params(refine_init=1)
    Z, labels, modes, st = slk.solve(dev(X), L, k, lam, dev(seeds), sigma=sig, params=p)
    np.testing.assert_array_equal(host(modes), ref["modes"])
    np.testing.assert_array_equal(host(labels), ref["labels"])
    assert np.abs(host(Z) - ref["Z"]).max() <= 1e-5
    assert st["energy"] == pytest.approx(ref["E"], rel=1e-6)


# ------------------------------------------------------------ K-means++ seeds

@pytest.mark.parametrize("case", ["blobs", "mixture", "mnist_like", "manifolds", "duplicates"])
def test_kmeanspp_matches_oracle(slk, case):
    """GPU K-means++ from the same draws gives the oracle's seeds index for
    index (and the numpy recipe's)."""
    if case == "blobs":
        X, _ = inputs.blobs()
        L, seed = 5, 1810
    elif case == "mixture":
        X, _ = inputs.mixture(20000, 9, 50, seed=8)
        L, seed = 50, 8
    elif case == "mnist_like":
        X, _ = inputs.mnist_like(N=6000)
        L, seed = 10, 1810
    elif case == "manifolds":
        X, _ = inputs.manifolds(N=20000)
        L, seed = 100, 1810
    else:   # every point repeated: exact zero distances, and an all-zero draw
        base = inputs.rng(3).normal(size=(7, 5)).astype(np.float32)
        X = np.repeat(base, 40, axis=0)
        L, seed = 12, 3
    first, u = inputs.kmeanspp_draws(X.shape[0], L, seed)
    want = oracle.kmeanspp(X, L, first, u)
    got = slk.kmeanspp(torch.from_numpy(X).cuda(), L, first, u).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got, inputs.kmeanspp(X, L, seed=seed))


def test_kmeanspp_rejects_bad_draws(slk):
    X = torch.zeros(10, 3, device="cuda")
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.kmeanspp(X, 3, 0, [0.5, 1.0])
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.kmeanspp(X, 3, 10, [0.5, 0.5])
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.kmeanspp(X, 11, 0, [0.5] * 10)
