"""Plain FP64 CPU oracle for K-means++ seeding in a kernel's feature space.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import or call this module; the CUDA library never imports it.

Sec. 2.1 of the paper names K-means++ as the initialization that samples each next initial
centroid from a weighted distribution favouring points far from those already chosen.  The
weighting of the cited method is the squared distance to the nearest chosen point, here taken
in the feature space of the kernel (the space Kernel K-means clusters in, Sec. 3):

    D(i) = min over chosen c of ||phi(p_i) - phi(p_c)||^2 = min_c (K_ii - 2 K_ic + K_cc).

``kmeanspp(K, k, u)`` takes the caller's k uniform draws u in [0, 1) (the random numbers are
inputs, so that the CUDA path and this oracle can be compared draw for draw):

* the first point is c_0 = floor(u_0 n) (uniform over the points);
* for t >= 1, with W = sum_i D(i): c_t is the point i at which the running sum of D over the
  points in index order first exceeds u_t W -- the inverse of the cumulative distribution of
  "i with probability D(i) / W"; if W = 0 (every point coincides with a chosen one), c_t =
  floor(u_t n);
* each point's initial label is the index t of its nearest chosen point (the lowest t on
  ties): the labels Kernel K-means starts from.

Pins (tests/test_oracle_seeding.py): the sampling law measured by sweeping a draw over [0, 1)
against D(i) / W computed from coordinates (linear kernel) and from an explicit degree-2
polynomial feature map; the degenerate W = 0 case; distinct centers that label themselves.
"""
from __future__ import annotations

import numpy as np

__all__ = ["kmeanspp"]


def _sqdist_to(K: np.ndarray, diag: np.ndarray, c: int) -> np.ndarray:
    """||phi(p_i) - phi(p_c)||^2 = K_ii - 2 K_ic + K_cc for every i, clamped at 0 (rounding
    can dip below)."""
    return np.maximum(diag - 2.0 * K[:, c] + K[c, c], 0.0)


def _nearest(D: np.ndarray, dc: np.ndarray, closer: np.ndarray) -> np.ndarray:
    """The squared distance to the nearest chosen point, after point c joined the chosen."""
    return np.where(closer, dc, D)


def kmeanspp(K: np.ndarray, k: int, u) -> dict:
    """K-means++ seeding on a kernel matrix K (n x n, FP64) with draws u (k values in [0, 1)).

    Returns {"centers": k point indices in the order chosen, "labels": n initial labels,
    "D": each point's final squared feature-space distance to its nearest center}."""
    K = np.asarray(K, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    n = K.shape[0]
    if not (1 <= k <= n) or u.shape[0] < k:
        raise ValueError("need 1 <= k <= n and k draws")
    diag = np.diag(K).copy()

    def dist_to(c: int) -> np.ndarray:
        return _sqdist_to(K, diag, c)

    centers = [min(int(np.floor(u[0] * n)), n - 1)]
    D = dist_to(centers[0])
    labels = np.zeros(n, dtype=np.int64)
    for t in range(1, k):
        W = float(np.sum(D))
        if W > 0.0:
            running = np.cumsum(D)
            c = int(np.searchsorted(running, u[t] * W, side="right"))
            c = min(c, n - 1)
        else:
            c = min(int(np.floor(u[t] * n)), n - 1)
        centers.append(c)
        dc = dist_to(c)
        closer = dc < D
        labels[closer] = t
        D = _nearest(D, dc, closer)
    return {"centers": np.array(centers, dtype=np.int64), "labels": labels, "D": D}
