"""Plain FP64 CPU oracle for Kernel K-means (Popcorn, arXiv 2501.05587).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
this module.  The CUDA library never imports it, and it imports nothing from
the CUDA library: the two share only the seeded generators in ``synth``.

What it computes, in the paper's notation (Sec. 3):

* ``kernel_matrix`` -- K_ij = kappa(p_i, p_j) for the linear, polynomial
  (Sec. 3.2, polynomial kernel (gamma x.y + c)^r) and Gaussian
  (Sec. 3.2, exp(-gamma ||x - y||^2 / sigma^2)) kernels.  The Gaussian squared
  distance is summed from coordinate differences, never from the norm
  expansion of Eq. 12 ("gauss"), so the oracle has no cancellation.
* ``selection_matrix`` -- V of Eq. 8 ("v_init"): V_ji = 1/|L_j| if p_i is in L_j.
* ``distances`` -- D = -2 K V^T + P~ + C~ (Eq. 11, "dist_sp_1") with
  P~ from diag(K) (Sec. 3.3) and C~ from diag(V K V^T) (Eq. 13, "c_norm"),
  both written as dense matrix products: no one-nonzero-per-column shortcut.
  An empty cluster (|L_j| = 0) has no centroid; its column of D is +inf.
* ``step`` -- one pass of the loop body of Alg. 2: D from the current labels,
  the row argmin (ties to the lowest cluster index), the objective
  J = sum_i D_{i, cl(i)} (the K-means objective of Sec. 2.1 in feature space),
  and per-row margins used by the parity rule.
* ``fit`` -- the loop of Alg. 2.  The paper's loop condition ("while the
  centroids are changing", Alg. 1/2) is read as: the centroids depend only on
  the labels, so the loop stops after a pass that changes no label (when
  convergence checking is on), or after a pass whose objective drop is at most
  tol * |J| (tol > 0), and always after max_iter passes.  The returned
  objective is J(labels_out).

Pins (tests/test_oracle_*.py): brute force over all labelings for n <= 8,
the linear kernel against Lloyd's algorithm in input space (Sec. 2.1), the
degree-2 polynomial kernel against Lloyd on an explicit feature map,
hand-derived golden cases (tests/golden/), kernel closed forms and invariants
(symmetry, Gaussian diagonal 1, monotone objective), and hand-worked rows for
the ``margin`` / ``scale`` outputs of ``step`` (a best-distance tie, k = 1, an
empty cluster, a singleton with D = 0).  No function here is "parity unpinned".
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "kernel_matrix",
    "selection_matrix",
    "distances",
    "step",
    "objective",
    "fit",
    "KIND_LINEAR",
    "KIND_POLYNOMIAL",
    "KIND_GAUSSIAN",
]

KIND_LINEAR = "linear"
KIND_POLYNOMIAL = "polynomial"
KIND_GAUSSIAN = "gaussian"


def _as64(P) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(P, dtype=np.float64))


def _sqdist_rows(Pa: np.ndarray, Pb: np.ndarray, block: int = 256) -> np.ndarray:
    """||a_i - b_j||^2 summed coordinate by coordinate (no norm expansion)."""
    out = np.empty((Pa.shape[0], Pb.shape[0]), dtype=np.float64)
    for i0 in range(0, Pa.shape[0], block):
        a = Pa[i0:i0 + block]
        acc = np.zeros((a.shape[0], Pb.shape[0]), dtype=np.float64)
        for l in range(Pa.shape[1]):
            diff = a[:, l:l + 1] - Pb[None, :, l]
            acc += diff * diff
        out[i0:i0 + block] = acc
    return out


def kernel_matrix(P, kern: dict, Q=None) -> np.ndarray:
    """K_ij = kappa(p_i, q_j) in FP64 (Q defaults to P, giving the n x n kernel matrix).

    Linear: p.q.  Polynomial (Sec. 3.2): (gamma p.q + c)^r with integer r >= 1,
    by repeated multiplication.  Gaussian (Sec. 3.2): exp(-gamma ||p-q||^2 / sigma^2),
    with gamma = 1 unless given.
    """
    Pa = _as64(P)
    Pb = Pa if Q is None else _as64(Q)
    kind = kern["kind"]
    if kind == KIND_LINEAR:
        return Pa @ Pb.T
    if kind == KIND_POLYNOMIAL:
        gamma = float(kern.get("gamma", 1.0))
        c = float(kern.get("coef0", 1.0))
        r = int(kern.get("degree", 2))
        if r < 1:
            raise ValueError("polynomial degree must be >= 1")
        base = gamma * (Pa @ Pb.T) + c
        out = base.copy()
        for _ in range(r - 1):
            out *= base
        return out
    if kind == KIND_GAUSSIAN:
        gamma = float(kern.get("gamma", 1.0))
        sigma = float(kern["sigma"])
        if sigma <= 0:
            raise ValueError("sigma must be > 0")
        return np.exp(-gamma * _sqdist_rows(Pa, Pb) / (sigma * sigma))
    raise ValueError(f"unknown kernel kind {kind!r}")


def selection_matrix(labels, k: int) -> np.ndarray:
    """Dense V (k x n) of Eq. 8: V_ji = 1/|L_j| where p_i is in L_j, else 0."""
    labels = np.asarray(labels, dtype=np.int64)
    n = labels.shape[0]
    counts = np.bincount(labels, minlength=k).astype(np.float64)
    V = np.zeros((k, n), dtype=np.float64)
    nz = counts[labels] > 0
    V[labels[nz], np.nonzero(nz)[0]] = 1.0 / counts[labels[nz]]
    return V


def distances(K: np.ndarray, labels, k: int) -> dict:
    """D = -2 K V^T + P~ + C~ (Eq. 11) with P~ = diag(K) and C~ = diag(V K V^T) (Eq. 13).

    Returns D (n x k, +inf in the columns of empty clusters), E = K V^T,
    the centroid norms cnorm_j = ||c_j||^2 and the counts |L_j|.
    """
    K = np.asarray(K, dtype=np.float64)
    labels = np.asarray(labels, dtype=np.int64)
    V = selection_matrix(labels, k)
    counts = np.bincount(labels, minlength=k)
    E = K @ V.T                          # (K V^T)_{ij} = <phi(p_i), c_j>
    cnorm = np.diag(V @ E)               # diag(V K V^T) = ||c_j||^2
    Ptil = np.diag(K)                    # ||phi(p_i)||^2
    D = -2.0 * E + Ptil[:, None] + cnorm[None, :]
    empty = counts == 0
    if empty.any():
        D[:, empty] = np.inf
    return {"D": D, "E": E, "cnorm": cnorm, "counts": counts, "kdiag": Ptil}


def objective(K: np.ndarray, labels, k: int) -> float:
    """J = sum_i ||phi(p_i) - c_{cl(i)}||^2 = sum_i D_{i, cl(i)}."""
    labels = np.asarray(labels, dtype=np.int64)
    D = distances(K, labels, k)["D"]
    return float(D[np.arange(labels.shape[0]), labels].sum())


def step(K: np.ndarray, labels, k: int) -> dict:
    """One loop body of Alg. 2: distances from ``labels``, row argmin, objective J(labels).

    Ties go to the lowest cluster index (np.argmin returns the first minimum).
    ``margin_i`` = second-smallest minus smallest D in row i (inf when k == 1 or
    only one cluster is non-empty); ``scale_i`` = max(|min_c D_ic|, K_ii).
    """
    labels = np.asarray(labels, dtype=np.int64)
    r = distances(K, labels, k)
    D = r["D"]
    n = labels.shape[0]
    new = np.argmin(D, axis=1).astype(np.int32)
    J = float(D[np.arange(n), labels].sum())
    if k > 1:
        part = np.partition(D, 1, axis=1)
        d1, d2 = part[:, 0], part[:, 1]
        with np.errstate(invalid="ignore"):
            margin = np.where(np.isfinite(d2), d2 - d1, np.inf)
    else:
        d1 = D[:, 0]
        margin = np.full(n, np.inf)
    scale = np.maximum(np.abs(d1), r["kdiag"])
    changed = int((new != labels).sum())
    return {"labels": new, "J": J, "D": D, "E": r["E"], "cnorm": r["cnorm"], "counts": r["counts"],
            "margin": margin, "scale": scale, "changed": changed, "kdiag": r["kdiag"]}


def fit(K: np.ndarray, k: int, init_labels, max_iter: int, tol: float = 0.0,
        check_convergence: bool = True) -> dict:
    """The loop of Alg. 2 on a given kernel matrix.

    Pass t computes D from labels cl_t, records J_t = J(cl_t) and the number of
    labels that change, and moves to cl_{t+1} = argmin.  With convergence
    checking on, the loop stops after a pass that changes no label (the
    centroids depend only on the labels, so they stopped changing), or after a
    pass t >= 1 with J_{t-1} - J_t <= tol * |J_t| when tol > 0.  ``iterations``
    counts passes; ``objective`` is J(labels_out).
    """
    labels = np.asarray(init_labels, dtype=np.int64).copy()
    n = labels.shape[0]
    if not (1 <= k):
        raise ValueError("k must be >= 1")
    if labels.min(initial=0) < 0 or labels.max(initial=0) >= k:
        raise ValueError("init labels out of range")
    J_hist, changed_hist, steps = [], [], []
    it = 0
    converged = False
    while it < max_iter:
        st = step(K, labels, k)
        J_hist.append(st["J"])
        changed_hist.append(st["changed"])
        steps.append(st)
        labels = st["labels"].astype(np.int64)
        it += 1
        if check_convergence:
            if st["changed"] == 0:
                converged = True
                break
            if tol > 0 and len(J_hist) >= 2 and J_hist[-2] - J_hist[-1] <= tol * abs(J_hist[-1]):
                break
    J_out = objective(K, labels, k) if n else 0.0
    return {"labels": labels.astype(np.int32), "objective": J_out, "iterations": it,
            "J_history": J_hist, "changed_history": changed_hist, "converged": converged,
            "steps": steps}
