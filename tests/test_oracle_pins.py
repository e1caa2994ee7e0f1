"""Pins for the FP64 oracle: each checks it against something other than itself.

* closed forms of the kernels, evaluated element by element with ``math``;
* hand-derived worked examples (tests/golden/);
* linear kernel == Lloyd's algorithm in input space (Sec. 2.1), written here
  with explicit centroids;
* polynomial kernel of degree 2 == Lloyd on the explicit feature map;
* diag(V K V^T) (Eq. 13) == the double sum (1/m^2) sum_{i,j in L_c} K_ij;
* brute force over every labeling for n <= 8: the converged labels are stable,
  J matches a pure-Python evaluation of the feature-space objective, and the
  global minimum is at most the converged J and is itself stable;
* monotone objective and the stopping rules of the loop.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import kkmeans
import synth


def _kern(kind, **kw):
    base = {"kind": kind, "gamma": 1.0, "coef0": 1.0, "degree": 2, "sigma": 1.0}
    base.update(kw)
    return base


# ---------------------------------------------------------------- kernel closed forms

@pytest.mark.parametrize("kern", [
    _kern("linear"),
    _kern("polynomial", gamma=0.5, coef0=2.0, degree=3),
    _kern("polynomial", gamma=1.0, coef0=1.0, degree=2),
    _kern("gaussian", sigma=1.7),
    _kern("gaussian", sigma=0.5, gamma=2.0),
])
def test_kernel_matrix_matches_elementwise_definition(kern):
    P = synth.gaussian_blobs(7, 4, 2, seed=3, box=2.0)
    K = oracle.kernel_matrix(P, kern)
    Pl = P.astype(float).tolist()
    for i in range(7):
        for j in range(7):
            x, y = Pl[i], Pl[j]
            dot = sum(a * b for a, b in zip(x, y))
            if kern["kind"] == "linear":
                ref = dot
            elif kern["kind"] == "polynomial":
                ref = (kern["gamma"] * dot + kern["coef0"]) ** kern["degree"]
            else:
                sq = sum((a - b) ** 2 for a, b in zip(x, y))
                ref = math.exp(-kern["gamma"] * sq / kern["sigma"] ** 2)
            assert K[i, j] == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_kernel_invariants():
    P = synth.rings(300, seed=5, d_pad=8)
    Kg = oracle.kernel_matrix(P, _kern("gaussian", sigma=0.5))
    assert np.array_equal(Kg, Kg.T)
    assert np.all(np.diag(Kg) == 1.0)
    assert np.all(Kg > 0) or np.all(Kg >= 0)
    assert np.all(Kg <= 1.0)
    Pi = synth.small_integer_points(50, 6, seed=1)
    Kp = oracle.kernel_matrix(Pi, _kern("polynomial", gamma=1.0, coef0=1.0, degree=2))
    assert np.array_equal(Kp, Kp.T)
    assert np.all(Kp == np.round(Kp))          # small integers: exact in FP64
    Kl = oracle.kernel_matrix(Pi, _kern("linear"))
    assert np.array_equal(Kl, Pi.astype(np.int64) @ Pi.astype(np.int64).T)


def test_gaussian_has_no_cancellation_for_near_duplicates():
    # two points 1e-6 apart at radius 1e3: the norm expansion would lose the distance entirely
    P = np.array([[1000.0, 0.0], [1000.0, 1e-3]], dtype=np.float32)
    K = oracle.kernel_matrix(P, _kern("gaussian", sigma=1e-3))
    d2 = float((np.float64(P[0, 1]) - np.float64(P[1, 1])) ** 2)
    assert K[0, 1] == pytest.approx(math.exp(-d2 / 1e-6), rel=1e-12)


# ---------------------------------------------------------------- hand-derived golden cases

def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def test_golden_linear_two_passes(golden_dir):
    g = _load(golden_dir, "linear_1d_two_passes.json")
    K = oracle.kernel_matrix(np.array(g["points"]), g["kernel"])
    st = oracle.step(K, g["labels"], g["k"])
    p1 = g["pass1"]
    np.testing.assert_allclose(st["E"], p1["E"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(st["cnorm"], p1["cnorm"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(st["D"], p1["D"], rtol=0, atol=1e-12)
    assert st["J"] == pytest.approx(p1["J"], abs=1e-12)
    assert st["labels"].tolist() == p1["new_labels"]
    assert st["changed"] == p1["changed"]
    f = g["fit"]
    r = oracle.fit(K, g["k"], g["labels"], f["max_iter"], check_convergence=f["check_convergence"])
    assert r["iterations"] == f["iterations"]
    assert r["objective"] == pytest.approx(f["objective"], abs=1e-12)
    assert r["labels"].tolist() == f["labels"]
    np.testing.assert_allclose(r["J_history"], f["J_history"], atol=1e-12)
    assert r["changed_history"] == f["changed_history"]


def test_golden_poly2(golden_dir):
    g = _load(golden_dir, "poly2_1d.json")
    K = oracle.kernel_matrix(np.array(g["points"]), g["kernel"])
    np.testing.assert_array_equal(K, np.array(g["K"], dtype=float))
    st = oracle.step(K, g["labels"], g["k"])
    p1 = g["pass1"]
    np.testing.assert_allclose(st["E"], p1["E"], atol=1e-12)
    np.testing.assert_allclose(st["cnorm"], p1["cnorm"], atol=1e-12)
    np.testing.assert_allclose(st["D"], p1["D"], atol=1e-12)
    assert st["J"] == pytest.approx(p1["J"], abs=1e-12)
    assert st["labels"].tolist() == p1["new_labels"]


def test_gaussian_closed_form_three_points():
    # x = [0, 1, 3], sigma = 1: K_01 = e^-1, K_02 = e^-9, K_12 = e^-4; labels [0, 0, 1]
    P = np.array([[0.0], [1.0], [3.0]])
    K = oracle.kernel_matrix(P, _kern("gaussian", sigma=1.0))
    st = oracle.step(K, [0, 0, 1], 2)
    e1, e4, e9 = math.exp(-1), math.exp(-4), math.exp(-9)
    c0 = (2 + 2 * e1) / 4.0
    assert st["cnorm"][0] == pytest.approx(c0, rel=1e-14)
    assert st["cnorm"][1] == pytest.approx(1.0, rel=1e-14)
    assert st["D"][2, 0] == pytest.approx(1 - (e9 + e4) + c0, rel=1e-14)
    assert st["D"][0, 1] == pytest.approx(1 - 2 * e9 + 1, rel=1e-14)
    assert st["D"][2, 1] == pytest.approx(0.0, abs=1e-15)
    assert st["J"] == pytest.approx(2 * (1 - (1 + e1) + c0) + 0.0, rel=1e-13)


# ---------------------------------------------------------------- Lloyd equivalences

def lloyd_step(X, labels, k):
    """Lloyd's three phases in an explicit space: means, squared distances, argmin."""
    X = np.asarray(X, dtype=np.float64)
    labels = np.asarray(labels)
    cents = np.zeros((k, X.shape[1]))
    empty = np.zeros(k, bool)
    for c in range(k):
        mem = X[labels == c]
        if len(mem) == 0:
            empty[c] = True
        else:
            cents[c] = mem.mean(axis=0)
    D = ((X[:, None, :] - cents[None, :, :]) ** 2).sum(axis=2)
    D[:, empty] = np.inf
    J = float(D[np.arange(len(labels)), labels].sum())
    return np.argmin(D, axis=1), J, D


def poly2_feature_map(X, gamma, c):
    """phi with <phi(x), phi(y)> = (gamma x.y + c)^2: (c, sqrt(2c gamma) x_l, gamma x_l^2, sqrt2 gamma x_l x_m)."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    cols = [np.full(n, c)]
    cols += [math.sqrt(2 * c * gamma) * X[:, l] for l in range(d)]
    cols += [gamma * X[:, l] ** 2 for l in range(d)]
    cols += [math.sqrt(2) * gamma * X[:, l] * X[:, m] for l in range(d) for m in range(l + 1, d)]
    return np.stack(cols, axis=1)


def _compare_trajectory(K, Phi, k, labels, steps, rtol=1e-9):
    for _ in range(steps):
        st = oracle.step(K, labels, k)
        ref_new, ref_J, ref_D = lloyd_step(Phi, labels, k)
        fin = np.isfinite(ref_D)
        np.testing.assert_allclose(st["D"][fin], ref_D[fin], rtol=rtol, atol=rtol * np.abs(ref_D[fin]).max())
        assert st["J"] == pytest.approx(ref_J, rel=rtol)
        safe = st["margin"] > 1e-9 * st["scale"]
        assert np.array_equal(st["labels"][safe], ref_new[safe])
        labels = st["labels"]
    return labels


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linear_kernel_is_lloyd_in_input_space(seed):
    X = synth.gaussian_blobs(240, 3, 5, seed=seed, box=4.0)
    k = 5
    K = oracle.kernel_matrix(X, _kern("linear"))
    lab = synth.init_labels(240, k, seed=100 + seed)
    _compare_trajectory(K, X, k, lab, steps=6)


@pytest.mark.parametrize("gamma,c", [(1.0, 1.0), (0.5, 2.0)])
def test_poly2_kernel_is_lloyd_on_explicit_feature_map(gamma, c):
    X = synth.gaussian_blobs(150, 3, 4, seed=7, box=2.0)
    Phi = poly2_feature_map(X, gamma, c)
    K = oracle.kernel_matrix(X, _kern("polynomial", gamma=gamma, coef0=c, degree=2))
    np.testing.assert_allclose(K, Phi @ Phi.T, rtol=1e-12, atol=1e-12)
    lab = synth.init_labels(150, 4, seed=9)
    _compare_trajectory(K, Phi, 4, lab, steps=5)


def test_cnorm_equals_double_sum():
    X = synth.gaussian_blobs(40, 3, 3, seed=4, box=2.0)
    K = oracle.kernel_matrix(X, _kern("gaussian", sigma=1.3))
    lab = synth.init_labels(40, 5, seed=5)
    r = oracle.distances(K, lab, 5)
    for c in range(5):
        mem = [i for i in range(40) if lab[i] == c]
        if not mem:
            continue
        ref = sum(K[i, j] for i in mem for j in mem) / len(mem) ** 2
        assert r["cnorm"][c] == pytest.approx(ref, rel=1e-13)


def test_empty_cluster_gets_infinite_distance():
    X = synth.gaussian_blobs(20, 2, 2, seed=1)
    K = oracle.kernel_matrix(X, _kern("linear"))
    lab = np.zeros(20, np.int32)
    lab[10:] = 2                       # cluster 1 empty
    st = oracle.step(K, lab, 3)
    assert np.all(np.isinf(st["D"][:, 1]))
    assert np.all(st["labels"] != 1)


# ---------------------------------------------------------------- brute force

def _pure_objective(K, labels, k):
    """sum_i ||phi(p_i) - c_{cl(i)}||^2 expanded by the kernel trick, in plain loops."""
    n = len(labels)
    J = 0.0
    for c in range(k):
        mem = [i for i in range(n) if labels[i] == c]
        m = len(mem)
        if m == 0:
            continue
        ss = sum(K[a][b] for a in mem for b in mem) / (m * m)
        for i in mem:
            J += K[i][i] - 2.0 * sum(K[i][j] for j in mem) / m + ss
    return J


def _pure_stable(K, labels, k, eps=1e-12):
    n = len(labels)
    mems = [[i for i in range(n) if labels[i] == c] for c in range(k)]
    ss = [sum(K[a][b] for a in m for b in m) / len(m) ** 2 if m else None for m in mems]
    for i in range(n):
        def dist(c):
            m = mems[c]
            return K[i][i] - 2.0 * sum(K[i][j] for j in m) / len(m) + ss[c]
        own = dist(labels[i])
        for c in range(k):
            if mems[c] and dist(c) < own - eps * max(1.0, abs(own)):
                return False
    return True


@pytest.mark.parametrize("n,k,kern,seed", [
    (7, 2, _kern("linear"), 0),
    (7, 3, _kern("polynomial", gamma=1.0, coef0=1.0, degree=2), 1),
    (8, 2, _kern("gaussian", sigma=1.0), 2),
    (6, 3, _kern("gaussian", sigma=0.7), 3),
])
def test_bruteforce_all_labelings(n, k, kern, seed):
    X = synth.gaussian_blobs(n, 2, k, seed=seed, box=2.0)
    K = oracle.kernel_matrix(X, kern)
    Kl = K.tolist()
    best_J, best_lab = math.inf, None
    for lab in itertools.product(range(k), repeat=n):
        J = _pure_objective(Kl, lab, k)
        if J < best_J:
            best_J, best_lab = J, lab
    assert _pure_stable(Kl, best_lab, k)                     # the global minimiser is Lloyd-stable
    for s in range(4):
        init = synth.init_labels(n, k, seed=50 + s)
        r = oracle.fit(K, k, init, max_iter=100, check_convergence=True)
        assert r["converged"]
        lab = r["labels"].tolist()
        assert r["objective"] == pytest.approx(_pure_objective(Kl, lab, k), rel=1e-12, abs=1e-12)
        assert _pure_stable(Kl, lab, k)                      # a local optimum of Lloyd's iteration
        assert best_J <= r["objective"] + 1e-12 * max(1.0, abs(best_J))


# ---------------------------------------------------------------- loop semantics

@pytest.mark.parametrize("kern", [_kern("gaussian", sigma=0.5), _kern("polynomial")])
def test_objective_non_increasing_and_fixed_point(kern):
    X = synth.rings(400, seed=3, d_pad=2) if kern["kind"] == "gaussian" else \
        synth.gaussian_blobs(400, 4, 6, seed=3, box=3.0)
    K = oracle.kernel_matrix(X, kern)
    r = oracle.fit(K, 6, synth.init_labels(400, 6, seed=4), max_iter=200, check_convergence=True)
    J = np.array(r["J_history"])
    assert np.all(np.diff(J) <= 1e-12 * np.abs(J[1:]))
    assert r["converged"]
    again = oracle.step(K, r["labels"], 6)
    assert again["changed"] == 0
    assert r["objective"] == pytest.approx(J[-1], rel=1e-13)


def test_fixed_iteration_mode_and_zero_iterations():
    X = synth.gaussian_blobs(100, 3, 3, seed=1)
    K = oracle.kernel_matrix(X, _kern("linear"))
    init = synth.init_labels(100, 3, seed=2)
    r0 = oracle.fit(K, 3, init, max_iter=0)
    assert r0["iterations"] == 0 and np.array_equal(r0["labels"], init)
    assert r0["objective"] == pytest.approx(oracle.objective(K, init, 3))
    r = oracle.fit(K, 3, init, max_iter=25, check_convergence=False)
    assert r["iterations"] == 25
    assert r["changed_history"][-1] == 0


def test_tolerance_stop():
    X = synth.gaussian_blobs(300, 3, 6, seed=8, box=3.0)
    K = oracle.kernel_matrix(X, _kern("linear"))
    init = synth.init_labels(300, 6, seed=9)
    full = oracle.fit(K, 6, init, max_iter=100)
    loose = oracle.fit(K, 6, init, max_iter=100, tol=1e-1)
    assert loose["iterations"] <= full["iterations"]
    Jh = loose["J_history"]
    if loose["iterations"] < full["iterations"]:
        assert Jh[-2] - Jh[-1] <= 1e-1 * abs(Jh[-1])


# ---------------------------------------------------------------- margin and scale of a step
#
# Every GPU parity test excuses a label mismatch only where the oracle's margin
# (second-best minus best distance of the row) is below 1e-6 times its scale
# max(|best D|, K_ii).  These pins fix both outputs on rows worked out by hand
# with the linear kernel in one dimension, where D_ic = (x_i - mean of cluster c)^2
# and every value below is a dyadic rational, exact in FP64.

MARGIN_CASES = [
    # points, labels, k, expected margin per row, expected scale per row, expected new labels
    # centroids 0.5, 6.5, 20 (a singleton); cluster 3 empty (its D column is +inf)
    ([0.0, 1.0, 3.0, 10.0, 20.0], [0, 0, 1, 1, 2], 4,
     [42.0, 30.0, 6.0, 78.0, 182.25],          # e.g. x=10: D = (90.25, 12.25, 100, inf)
     [0.25, 1.0, 9.0, 100.0, 400.0],           # x=20: best D = 0 (singleton), floored by K_ii = 400
     [0, 0, 0, 1, 2]),
    # k = 1: no second cluster, margin +inf; scale = max(|D|, K_ii), D = (1, 1)
    ([0.0, 2.0], [0, 0], 1, [math.inf, math.inf], [1.0, 4.0], [0, 0]),
    # k = 2 with one cluster empty: the second-best is +inf, so the margin is +inf
    ([0.0, 2.0], [0, 0], 2, [math.inf, math.inf], [1.0, 4.0], [0, 0]),
    # centroids 0, 2, 5.5: x = 1 is equidistant from clusters 0 and 1 (margin 0, tie to 0)
    ([0.0, 2.0, 1.0, 10.0], [0, 1, 2, 2], 3,
     [4.0, 4.0, 0.0, 64.0 - 20.25],            # x=0: D = (0, 4, 30.25); x=10: D = (100, 64, 20.25)
     [0.0, 4.0, 1.0, 100.0],                    # x=0: best D = 0 and K_ii = 0
     [0, 1, 0, 2]),
]


def margin_pins_hold(step_fn) -> bool:
    """True when step_fn reproduces every hand-worked margin, scale and label above."""
    for pts, lab, k, margin, scale, new in MARGIN_CASES:
        K = oracle.kernel_matrix(np.array(pts)[:, None], _kern("linear"))
        st = step_fn(K, lab, k)
        m = np.asarray(st["margin"], dtype=float)
        s = np.asarray(st["scale"], dtype=float)
        if not np.array_equal(np.isinf(m), np.isinf(np.array(margin))):
            return False
        fin = np.isfinite(margin)
        if not np.allclose(m[fin], np.array(margin)[fin], rtol=0, atol=1e-12):
            return False
        if not np.allclose(s, scale, rtol=0, atol=1e-12):
            return False
        if st["labels"].tolist() != new:
            return False
    return True


def test_step_margin_and_scale_hand_worked():
    assert margin_pins_hold(oracle.step)


def test_parity_exemption_uses_margin_and_scale():
    """The parity rule excuses a flipped label only on a near-tie row: on the tied row of
    the last case a GPU label of 1 is exempt; on every other row a flip is not."""
    from tests.parity import label_mismatches

    pts, lab, k = [0.0, 2.0, 1.0, 10.0], [0, 1, 2, 2], 3
    K = oracle.kernel_matrix(np.array(pts)[:, None], _kern("linear"))
    st = oracle.step(K, lab, k)
    assert label_mismatches([0, 1, 1, 2], st) == (0, 1)      # the tie: exempt
    assert label_mismatches([1, 1, 0, 2], st) == (1, 0)      # margin 4 on scale 0 -> 4 > 0: not exempt
    assert label_mismatches([0, 1, 0, 1], st) == (1, 0)
