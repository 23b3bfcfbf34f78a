"""slk_bound_iterate_noalloc: the z-updates for callers that cannot allocate
device memory (a plug-in inside a framework that has reserved the device
memory for its own pool, or a serving loop that may not allocate after
start-up).  Its scratch is a static device array inside the library, so it is
checked against the allocating entry point slk_bound_iterate, on two calls in
a row (the second call runs on the array the first one left behind).

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1810_13044_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Z_TOL = 1e-5   # the Z tolerance of the parity tests


@pytest.fixture(scope="module")
def slk():
    from paper_1810_13044_gb300 import build, slk as _slk
    build.build()
    return _slk


def _case(N, L, k, weighted, seed):
    rp, ci, w = inputs.random_graph(N, k, seed=seed, weighted=weighted)
    A = inputs.random_unary(N, L, seed=seed + 1)
    Z0 = inputs.random_simplex_rows(N, L, seed=seed + 2)
    d = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return d(rp), d(ci), d(w), d(A), d(Z0)


def test_noalloc_matches_allocating_entry_point_twice(slk):
    cases = [  # (N, L, k, weighted, max_iters, tol): the 70000 x 784 workload's
        (70000, 10, 5, False, 7, -1.0),          # bound shape, then a ragged one
        (3001, 33, 6, True, 100, 1e-6),          # that stops on the tolerance
    ]
    for N, L, k, weighted, iters, tol in cases:
        rp, ci, w, A, Z0 = _case(N, L, k, weighted, seed=N + L)
        Z_ref, Zp = Z0.clone(), torch.empty_like(Z0)
        it_ref, dl_ref = slk.bound_iterate(A, rp, ci, w, 1.0, Z_ref, Zp, iters, tol=tol)
        Z_na = Z0.clone()
        it_na, dl_na = slk.bound_iterate_noalloc(A, rp, ci, w, 1.0, Z_na, iters, tol=tol)
        assert it_na == it_ref
        assert abs(dl_na - dl_ref) <= Z_TOL
        assert (Z_na - Z_ref).abs().max().item() <= Z_TOL


def test_noalloc_matches_oracle(slk):
    """The same z-updates against the FP64 oracle, within the Z tolerance."""
    N, L, k = 4000, 17, 5
    rp, ci, w = inputs.random_graph(N, k, seed=77, weighted=True)
    A = inputs.random_unary(N, L, seed=78)
    Z0 = inputs.random_simplex_rows(N, L, seed=79)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for iters in (1, 6):
        Z = d(Z0)
        it, _ = slk.bound_iterate_noalloc(d(A), d(rp), d(ci), d(w), 1.3, Z, iters, tol=-1.0)
        Zo, _, ito, _ = oracle.bound_iterate(A, rp, ci, w, 1.3, Z0, iters)
        assert it == ito == iters
        assert np.abs(Z.cpu().numpy() - Zo).max() <= Z_TOL


def test_noalloc_zero_iterations_leaves_z(slk):
    rp, ci, w, A, Z0 = _case(1000, 7, 4, False, seed=5)
    Z = Z0.clone()
    it, dl = slk.bound_iterate_noalloc(A, rp, ci, w, 1.0, Z, 0)
    assert it == 0 and dl == 0.0
    assert torch.equal(Z, Z0)


def test_noalloc_rejects_sizes_beyond_its_scratch(slk):
    N, L = slk.NOALLOC_MAX_ELEMS // 8 + 1, 8
    A = torch.zeros(N, L, device="cuda")
    Z = torch.full((N, L), 1.0 / L, device="cuda")
    rp = torch.arange(N + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(N, dtype=torch.int32, device="cuda")
    with pytest.raises(slk.SlkError, match="SCRATCH_LIMIT"):
        slk.bound_iterate_noalloc(A, rp, ci, None, 1.0, Z, 3)
