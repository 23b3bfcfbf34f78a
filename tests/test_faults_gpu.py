"""Failure detection without a GPU fault: the bounded waits of the
persistent z-update kernels give up and report SLK_ERR_TIMEOUT, and the
context keeps working afterwards."""
import time

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


def test_barrier_wait_gives_up_and_context_stays_usable(slk):
    """One block waits at the device-wide barrier for a block that is never
    launched (an arrival target nothing reaches): the wait ends after its
    limit with SLK_ERR_TIMEOUT, and the next z-updates on the same context
    run normally and match the oracle."""
    for timeout_ms in (20, 200):
        t0 = time.perf_counter()
        with pytest.raises(slk.SlkError, match="TIMEOUT"):
            slk.barrier_selftest(timeout_ms)
        elapsed = time.perf_counter() - t0
        assert timeout_ms / 1e3 <= elapsed < timeout_ms / 1e3 + 2.0
    N, L, k = 5000, 12, 6
    rp, ci, w = inputs.random_graph(N, k, seed=3, weighted=True)
    A = inputs.random_unary(N, L, seed=4)
    Z0 = inputs.random_simplex_rows(N, L, seed=5)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Z, Zp = d(Z0), torch.empty(N, L, device="cuda")
    it, _ = slk.bound_iterate(d(A), d(rp), d(ci), d(w), 1.0, Z, Zp, 9, tol=-1.0)
    Zo, _, ito, _ = oracle.bound_iterate(A, rp, ci, w, 1.0, Z0, 9)
    assert it == ito == 9
    assert np.abs(Z.cpu().numpy() - Zo).max() <= 1e-5


def test_barrier_selftest_rejects_bad_limits(slk):
    for bad in (0, -5, 2001):
        with pytest.raises(slk.SlkError, match="INVALID_ARG"):
            slk.barrier_selftest(bad)
