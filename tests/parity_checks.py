"""Comparison of a GPU solve with the FP64 oracle's, shared by the parity
tests.  Integer results are compared exactly, except where float rounding
decides them between near-equal values of the oracle's own result:

* a label p may differ only if the oracle's z_p of the two labels agree
  within the Z tolerance (e.g. a point far from every mode, whose unary
  terms underflow float32 to 0 while float64 still orders them);
* a mode l may differ only if the oracle's log z of the two points agree
  within KEY_TIE.

Such near-ties are counted and bounded by the caller."""
import numpy as np

Z_TOL = 1e-5
E_RTOL = 1e-6
KEY_TIE = 1e-5


def compare_solve(Z, labels, modes, stats, ref, max_label_ties=1e-3, max_mode_ties=None,
                  energy_at=None):
    """Z, labels, modes: numpy arrays of the GPU result; stats: its dict;
    ref: oracle.solve / solve_graph output.  When labels or modes differ (at
    near-ties), the discrete energy of Eq. (1) is no longer the same number
    on both sides; energy_at(labels, modes) -> the oracle's energy at the
    GPU's labels and modes is then the value the GPU's energy must match.
    Returns (mode ties, label ties, max |dZ|)."""
    Zo = ref["Z"]
    N, L = Zo.shape
    assert stats["outer_iters"] == ref["outer"], (stats["outer_iters"], ref["outer"])
    logZ = np.log(np.maximum(Zo, 1e-300))
    gm, om = np.asarray(modes), ref["modes"]
    mode_ties = 0
    for l in np.nonzero(gm != om)[0]:
        assert abs(logZ[gm[l], l] - logZ[om[l], l]) <= KEY_TIE, (l, gm[l], om[l])
        mode_ties += 1
    if max_mode_ties is not None:
        assert mode_ties <= max_mode_ties, mode_ties
    gl, ol = np.asarray(labels), ref["labels"]
    bad = np.nonzero(gl != ol)[0]
    for p in bad:
        assert abs(Zo[p, gl[p]] - Zo[p, ol[p]]) <= Z_TOL, (p, gl[p], ol[p])
    assert bad.size <= max(1, int(max_label_ties * N)), bad.size
    err = float(np.abs(np.asarray(Z, dtype=np.float64) - Zo).max())
    assert err <= Z_TOL, err
    E = stats["energy"]
    E_ref = ref["E"]
    if (mode_ties or bad.size) and energy_at is not None:
        E_ref = energy_at(gl, gm)
    assert abs(E - E_ref) <= E_RTOL * abs(E_ref), (E, E_ref, ref["E"])
    return mode_ties, int(bad.size), err
