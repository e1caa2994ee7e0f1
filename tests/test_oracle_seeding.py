"""Pins for the K-means++ seeding oracle (oracle/seeding.py), CPU only.

The oracle takes the caller's draws, so its sampling law can be measured exactly: sweeping
the draw u_t over a fine grid of [0, 1) with the earlier draws fixed, the fraction of the
grid that selects point i must be D(i) / W, where D(i) is the squared distance from point i
to its nearest chosen point.  Here D is computed independently of the oracle's kernel-matrix
arithmetic: from coordinates for the linear kernel (input space, Sec. 2.1) and from an
explicit degree-2 feature map for the polynomial kernel.  A mistake in the weights (D
instead of D^2, the wrong center, a dropped K_cc), in the cumulative order or in the
boundary rule moves these fractions.  Also pinned: the degenerate case where every point
coincides (uniform fallback), distinct centers, each center labelled by itself, and every
label being the nearest chosen point.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle.seeding import kmeanspp

GRID = 20000


def _poly2_features(X, gamma=1.0, c=1.0):
    """phi with phi(x).phi(y) = (gamma x.y + c)^2: (c, sqrt(2 c gamma) x_l, gamma x_l^2,
    sqrt(2) gamma x_l x_m for l < m)."""
    cols = [np.full(len(X), c), *(np.sqrt(2 * c * gamma) * X.T), *(gamma * X.T ** 2)]
    for l, m in itertools.combinations(range(X.shape[1]), 2):
        cols.append(np.sqrt(2.0) * gamma * X[:, l] * X[:, m])
    return np.stack(cols, axis=1)


def _sweep(K, k, u_fixed):
    """Fraction of a grid of the last draw that selects each point as the k-th center."""
    n = K.shape[0]
    counts = np.zeros(n)
    for g in range(GRID):
        u = np.concatenate([u_fixed, [(g + 0.5) / GRID]])
        counts[kmeanspp(K, k, u)["centers"][-1]] += 1
    return counts / GRID


@pytest.mark.parametrize("space", ["linear", "poly2"])
def test_sampling_law_is_squared_distance_to_nearest_center(space):
    rng = np.random.default_rng(7)
    X = rng.normal(size=(9, 2))
    if space == "linear":
        K = oracle.kernel_matrix(X, {"kind": "linear"})
        F = X                                             # input space
    else:
        kern = {"kind": "polynomial", "gamma": 1.0, "coef0": 1.0, "degree": 2}
        K = oracle.kernel_matrix(X, kern)
        F = _poly2_features(X)                            # explicit feature space
    sq = ((F[:, None, :] - F[None, :, :]) ** 2).sum(-1)   # squared distances, from coordinates
    u0 = 0.41                                             # first center: floor(0.41 * 9) = 3
    c0 = 3
    frac = _sweep(K, 2, [u0])
    D = sq[:, c0]
    np.testing.assert_allclose(frac, D / D.sum(), atol=2.0 / GRID)
    assert frac[c0] == 0.0
    # third center given the first two: weights min(distance to c0, distance to c1)
    u1 = 0.77
    c1 = kmeanspp(K, 2, [u0, u1])["centers"][1]
    frac3 = _sweep(K, 3, [u0, u1])
    D2 = np.minimum(sq[:, c0], sq[:, c1])
    np.testing.assert_allclose(frac3, D2 / D2.sum(), atol=2.0 / GRID)


def test_labels_are_the_nearest_chosen_point_and_centers_are_distinct():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(60, 3))
    K = oracle.kernel_matrix(X, {"kind": "linear"})
    u = rng.random(6)
    r = kmeanspp(K, 6, u)
    c = r["centers"]
    assert len(set(c.tolist())) == 6
    assert np.array_equal(r["labels"][c], np.arange(6))
    sq = ((X[:, None, :] - X[None, c, :]) ** 2).sum(-1)   # to each chosen point, from coordinates
    np.testing.assert_array_equal(r["labels"], np.argmin(sq, axis=1))
    np.testing.assert_allclose(r["D"], sq.min(axis=1), rtol=1e-12, atol=1e-12)


def test_first_center_is_uniform_and_coincident_points_fall_back_to_uniform():
    X = np.ones((10, 2))                                  # every point the same: W = 0 after c0
    K = oracle.kernel_matrix(X, {"kind": "gaussian", "gamma": 1.0, "sigma": 1.0})
    r = kmeanspp(K, 3, [0.05, 0.55, 0.95])
    assert r["centers"].tolist() == [0, 5, 9]
    assert np.all(r["labels"] == 0)                       # ties go to the lowest index


# ---------------------------------------------------------------- planted mistakes

def _mut_distance_not_squared(K, diag, c):
    return np.sqrt(np.maximum(diag - 2.0 * K[:, c] + K[c, c], 0.0))


def _mut_drop_kcc(K, diag, c):
    return np.maximum(diag - 2.0 * K[:, c], 0.0)


@pytest.mark.parametrize("which", ["distance_not_squared", "drop_kcc", "last_center_only"])
def test_pins_catch_planted_mistakes(monkeypatch, which):
    """Each mutant of the seeding oracle must fail the sampling-law pin."""
    from oracle import seeding
    if which == "distance_not_squared":
        monkeypatch.setattr(seeding, "_sqdist_to", _mut_distance_not_squared)
    elif which == "drop_kcc":
        monkeypatch.setattr(seeding, "_sqdist_to", _mut_drop_kcc)
    else:
        monkeypatch.setattr(seeding, "_nearest", lambda D, dc, closer: dc)
    with pytest.raises(AssertionError):
        test_sampling_law_is_squared_distance_to_nearest_center("poly2")
