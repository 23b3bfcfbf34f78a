"""Batched form: many uneven problems in one slk_solve_batched call give the
same results as slk_solve on each problem alone (and as the FP64 oracle)."""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slk():
    from paper_1810_13044_gb300 import build, slk as _slk
    build.build()
    return _slk


def _problems(count, seed, n_range=(300, 3000), Ds=(9, 64, 256), L_range=(5, 50)):
    g = inputs.rng(seed)
    out = []
    for i in range(count):
        N = int(g.integers(*n_range))
        D = int(g.choice(Ds))
        L = int(g.integers(L_range[0], L_range[1] + 1))
        L = min(L, N // 4)
        X, _ = inputs.mixture(N, D, L, seed=seed * 1000 + i)
        m0 = inputs.kmeanspp(X, L, seed=seed * 1000 + i)
        out.append(dict(Xh=X, m0h=m0, X=torch.from_numpy(X).cuda(), L=L, k=5, lam=1.0,
                        init_modes=torch.from_numpy(m0).cuda()))
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16_rerank"])
def test_batched_equals_single(slk, precision):
    probs = _problems(12, seed=3)
    p = slk.default_params(knn_precision=precision)
    res = slk.solve_batched(probs, params=p)
    for pr, (Z, lab, modes, st) in zip(probs, res):
        Z1, lab1, modes1, st1 = slk.solve(pr["X"], pr["L"], pr["k"], pr["lam"], pr["init_modes"], params=p)
        assert st["outer_iters"] == st1["outer_iters"]
        assert st["inner_iters_total"] == st1["inner_iters_total"]
        assert torch.equal(modes, modes1)
        assert torch.equal(lab, lab1)
        assert (Z - Z1).abs().max().item() <= 1e-6
        assert st["energy"] == pytest.approx(st1["energy"], rel=1e-9)
        assert st["sigma"] == st1["sigma"]


def test_batched_matches_oracle(slk):
    """Well-separated blobs of different N, D, L: the batch members equal the
    oracle's solves.  (On mixtures whose K-means++ seeds leave clusters empty,
    an empty cluster's mode is a float32 near-tie among points with z ~ 1/L,
    so only the batched == single-problem check above applies there.)"""
    probs = []
    for i, (N, D, L) in enumerate([(400, 9, 3), (650, 16, 7), (300, 5, 4), (900, 12, 11)]):
        X, _ = inputs.blobs(N=N, D=D, n_blobs=L, seed=40 + i)
        m0 = inputs.kmeanspp(X, L, seed=40 + i)
        probs.append(dict(Xh=X, m0h=m0, X=torch.from_numpy(X).cuda(), L=L, k=5, lam=1.0,
                          init_modes=torch.from_numpy(m0).cuda()))
    res = slk.solve_batched(probs)
    for pr, (Z, lab, modes, st) in zip(probs, res):
        # both start from the batch member's sigma
        ref = oracle.solve(pr["Xh"], pr["L"], pr["k"], pr["lam"], pr["m0h"], sig=st["sigma"])
        np.testing.assert_array_equal(modes.cpu().numpy(), ref["modes"])
        np.testing.assert_array_equal(lab.cpu().numpy(), ref["labels"])
        assert np.abs(Z.cpu().numpy() - ref["Z"]).max() <= 1e-5
        assert st["energy"] == pytest.approx(ref["E"], rel=1e-6)


def test_batched_heat_affinity_and_single_problem(slk):
    probs = _problems(1, seed=9, n_range=(1000, 1001), Ds=(64,), L_range=(64, 64))
    p = slk.default_params(affinity="heat")
    (Z, lab, modes, st), = slk.solve_batched(probs, params=p)
    Z1, lab1, modes1, st1 = slk.solve(probs[0]["X"], probs[0]["L"], 5, 1.0, probs[0]["init_modes"], params=p)
    assert torch.equal(lab, lab1) and torch.equal(modes, modes1)
    assert (Z - Z1).abs().max().item() <= 1e-6


def test_batched_rejects_large_L(slk):
    probs = _problems(1, seed=11, n_range=(500, 501), Ds=(9,), L_range=(5, 5))
    probs[0]["L"] = 129
    probs[0]["init_modes"] = torch.arange(129, dtype=torch.int32, device="cuda")
    with pytest.raises(slk.SlkError, match="INVALID_ARG"):
        slk.solve_batched(probs)
