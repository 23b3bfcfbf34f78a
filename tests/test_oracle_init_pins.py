"""Pins of the starting-mode part of the FP64 oracle (Section 4.2: the
starting mode of each cluster follows the mode definition of Eq. (1) from
the initial, nearest-seed assignments).

Checked against: scipy's pairwise distances for the nearest-seed cells, the
symmetry of a one-dimensional cluster, the two limits of the kernel width
(very wide: the density is n - sum ||x_p - y||^2 / (2 sigma^2), so the mode
is the data point nearest the cluster mean; very narrow: a duplicated point
doubles its own density and wins), one-point and empty clusters.
"""
import numpy as np
import pytest

import oracle

spatial = pytest.importorskip("scipy.spatial")


def test_assignment_is_nearest_seed():
    g = np.random.default_rng(1)
    X = g.normal(size=(200, 5)).astype(np.float32)
    seeds = np.array([3, 50, 77, 120], np.int32)
    _, assign, _ = oracle.initial_modes(X, seeds, 1.0)
    d = spatial.distance.cdist(X.astype(np.float64), X[seeds].astype(np.float64), "sqeuclidean")
    np.testing.assert_array_equal(assign, np.argmin(d, axis=1))


def test_seed_ties_go_to_the_smaller_label_and_empty_cluster_keeps_its_seed():
    X = np.array([[0.0], [1.0], [2.0], [0.0], [7.0]], np.float32)
    seeds = np.array([0, 3, 4], np.int32)          # x_0 == x_3: label 1 gets no point
    modes, assign, dens = oracle.initial_modes(X, seeds, 1.0)
    assert list(assign) == [0, 0, 0, 0, 2]
    assert modes[1] == 3 and dens[1] == 0.0
    assert modes[2] == 4 and dens[2] == pytest.approx(1.0, abs=0)


def test_symmetric_cluster_mode_is_its_centre():
    # 9 equally spaced points, unimodal symmetric density: the middle point
    X = np.concatenate([np.arange(-4, 5, dtype=np.float32), [40.0, 41.0]])[:, None]
    seeds = np.array([0, 9], np.int32)             # seed at the left end of the cluster
    for sig in (0.7, 1.5, 3.0):
        modes, assign, _ = oracle.initial_modes(X, seeds, sig)
        assert list(assign[:9]) == [0] * 9
        assert modes[0] == 4


def test_wide_kernel_mode_is_point_nearest_the_mean():
    g = np.random.default_rng(7)
    X = np.concatenate([g.normal(0, 1, (60, 3)), g.normal(30, 1, (60, 3))]).astype(np.float32)
    seeds = np.array([5, 70], np.int32)
    modes, assign, _ = oracle.initial_modes(X, seeds, 1e3)
    X64 = X.astype(np.float64)
    for l in range(2):
        mean = X64[assign == l].mean(0)
        assert modes[l] == int(np.argmin(((X64 - mean) ** 2).sum(1)))


def test_narrow_kernel_duplicate_wins():
    g = np.random.default_rng(8)
    X = g.normal(size=(40, 4)).astype(np.float32)
    X[31] = X[12]                                  # a duplicate inside the cloud
    seeds = np.array([0], np.int32)
    modes, _, dens = oracle.initial_modes(X, seeds, 1e-3)
    assert modes[0] == 12
    assert dens[0] == pytest.approx(2.0, rel=1e-12)


def test_one_point_cluster_and_density_consistency():
    X = np.array([[0.0, 0.0], [0.5, 0.0], [1.0, 0.0], [50.0, 50.0]], np.float32)
    seeds = np.array([1, 3], np.int32)
    modes, assign, dens = oracle.initial_modes(X, seeds, 0.8)
    assert modes[1] == 3 and dens[1] == pytest.approx(1.0, abs=0)
    assert modes[0] == 1
    f = oracle.cluster_density(X, assign, 0, 0.8, np.arange(4))
    assert f[1] == pytest.approx(dens[0], rel=1e-15)
    assert np.argmax(f) == 1
    # the density of cluster 0 at x_1: 1 + 2 exp(-0.25 / (2 * 0.64))
    assert f[1] == pytest.approx(1.0 + 2.0 * np.exp(-0.25 / 1.28), rel=1e-14)
