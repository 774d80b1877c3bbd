"""Cluster labels of a colour field, and label agreement.

TEST INFRASTRUCTURE (see the package docstring): never imported by the CUDA path.

The paper segments its outputs with a watershed at threshold 0.02 (Section 5).  Here a
cluster is a connected component of the 4-neighbour pixel graph in which two neighbours
are joined when every channel differs by at most the threshold.  The label of a pixel
is the smallest row-major index in its component, a canonical form that two labelings
can be compared with directly.  The join decision is taken in float32, the precision
of the colour fields it is applied to: |fl32(a - b)| <= fl32(threshold).
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

THRESHOLD = 0.02


def _joins(c32: np.ndarray, thr: np.float32):
    """Boolean masks of joined horizontal (H, W-1) and vertical (H-1, W) neighbour pairs."""
    dh = np.max(np.abs(c32[:, 1:, :] - c32[:, :-1, :]), axis=-1) <= thr
    dv = np.max(np.abs(c32[1:, :, :] - c32[:-1, :, :]), axis=-1) <= thr
    return dh, dv


def cluster_labels(c: np.ndarray, threshold: float = THRESHOLD):
    """Canonical component labels (H, W) int64 and the number of components; the
    components come from scipy's graph connected-components routine."""
    c32 = np.asarray(c).astype(np.float32)
    H, W, _ = c32.shape
    N = H * W
    dh, dv = _joins(c32, np.float32(threshold))
    idx = np.arange(N).reshape(H, W)
    a = np.concatenate([idx[:, :-1][dh], idx[:-1, :][dv]])
    b = np.concatenate([idx[:, 1:][dh], idx[1:, :][dv]])
    graph = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(N, N))
    ncomp, comp = connected_components(graph, directed=False)
    smallest = np.full(ncomp, N, dtype=np.int64)
    np.minimum.at(smallest, comp, np.arange(N))
    return smallest[comp].reshape(H, W), int(ncomp)


def cluster_labels_bfs(c: np.ndarray, threshold: float = THRESHOLD):
    """Brute-force breadth-first labelling (for small images); same canonical form."""
    c32 = np.asarray(c).astype(np.float32)
    H, W, _ = c32.shape
    thr = np.float32(threshold)
    lab = np.full((H, W), -1, dtype=np.int64)
    count = 0
    for start in range(H * W):
        r0, q0 = divmod(start, W)
        if lab[r0, q0] >= 0:
            continue
        count += 1
        lab[r0, q0] = start
        queue = deque([(r0, q0)])
        while queue:
            r, q = queue.popleft()
            for rr, qq in ((r - 1, q), (r + 1, q), (r, q - 1), (r, q + 1)):
                if 0 <= rr < H and 0 <= qq < W and lab[rr, qq] < 0:
                    if np.max(np.abs(c32[rr, qq] - c32[r, q])) <= thr:
                        lab[rr, qq] = start
                        queue.append((rr, qq))
    return lab, count


def label_agreement(a: np.ndarray, b: np.ndarray) -> float:
    """Fraction of pixels whose canonical labels are equal."""
    return float(np.mean(np.asarray(a) == np.asarray(b)))
