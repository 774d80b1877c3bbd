"""Pins for the oracle's cluster labels: brute-force BFS against the library
connected-components routine, and piecewise-constant images with known regions."""
import numpy as np

from oracle.labels import cluster_labels, cluster_labels_bfs, label_agreement


def test_blocks_known_regions():
    c = np.zeros((6, 8, 3))
    c[:, :3] = [0.1, 0.2, 0.3]
    c[:, 3:] = [0.6, 0.2, 0.3]
    c[3:, 5:] = [0.6, 0.2, 0.9]
    lab, n = cluster_labels(c)
    expect = np.zeros((6, 8), dtype=np.int64)
    expect[:, 3:] = 3
    expect[3:, 5:] = 3 * 8 + 5
    assert n == 3 and np.array_equal(lab, expect)


def test_threshold_is_inclusive_in_float32():
    a = np.float32(0.5)
    b = np.float32(a + np.float32(0.02))
    c = np.array([[[a], [b]]], dtype=np.float64)
    lab, n = cluster_labels(c)
    joined = abs(np.float32(b) - np.float32(a)) <= np.float32(0.02)
    assert (n == 1) == bool(joined)


def test_bfs_matches_library(rng):
    for trial in range(8):
        H, W, C = rng.integers(1, 12), rng.integers(1, 12), rng.integers(1, 4)
        # quantised colours so that many neighbours fall either side of the threshold
        c = np.round(rng.uniform(size=(H, W, C)) * 20) / 400.0
        lab1, n1 = cluster_labels(c)
        lab2, n2 = cluster_labels_bfs(c)
        assert n1 == n2 and np.array_equal(lab1, lab2)
        # canonical: each label is the smallest index of its component
        flat = lab1.reshape(-1)
        for l in np.unique(flat):
            assert np.min(np.nonzero(flat == l)[0]) == l


def test_agreement():
    a = np.arange(12).reshape(3, 4)
    b = a.copy()
    b[0, 0] = 99
    assert label_agreement(a, a) == 1.0
    assert label_agreement(a, b) == 11 / 12
