"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Each mutant replaces ``oracle.kkmeans.distances`` with a variant carrying one
mistake -- a dropped term, a wrong sign, a wrong scale in V, a wrong index --
and the pins of test_oracle_pins (golden case, Lloyd equivalence) are re-run
against it.  A mutant that no pin rejects would mean the pins are too weak.
"""
import numpy as np
import pytest

import oracle
from oracle import kkmeans
import synth
from tests.test_oracle_pins import lloyd_step, margin_pins_hold

_orig = kkmeans.distances
_orig_step = kkmeans.step


def _mut_drop_cnorm(K, labels, k):
    r = _orig(K, labels, k)
    D = r["D"] - r["cnorm"][None, :]
    return {**r, "D": D}


def _mut_sign_E(K, labels, k):
    r = _orig(K, labels, k)
    D = r["D"] + 4.0 * r["E"]
    return {**r, "D": D}


def _mut_V_counts(K, labels, k):
    # V_ji = |L_j| instead of 1/|L_j|
    labels = np.asarray(labels, dtype=np.int64)
    counts = np.bincount(labels, minlength=k).astype(float)
    V = np.zeros((k, len(labels)))
    V[labels, np.arange(len(labels))] = counts[labels]
    E = K @ V.T
    cnorm = np.diag(V @ E)
    D = -2 * E + np.diag(K)[:, None] + cnorm[None, :]
    D[:, counts == 0] = np.inf
    return {"D": D, "E": E, "cnorm": cnorm, "counts": counts.astype(int), "kdiag": np.diag(K)}


def _mut_factor_two(K, labels, k):
    r = _orig(K, labels, k)
    return {**r, "D": r["D"] + r["E"]}          # -E instead of -2E


def _mut_diag_index(K, labels, k):
    r = _orig(K, labels, k)
    return {**r, "D": r["D"] - np.diag(K)[:, None] + K[0, 0]}   # K_00 for every row


def _mut_transposed_V(K, labels, k):
    # uses the column index of K instead of the row: E = V K (k x n) transposed back, with a shifted label
    r = _orig(K, labels, k)
    E = np.roll(r["E"], 1, axis=0)
    D = -2 * E + np.diag(K)[:, None] + r["cnorm"][None, :]
    return {**r, "E": E, "D": D}


MUTANTS = [_mut_drop_cnorm, _mut_sign_E, _mut_V_counts, _mut_factor_two, _mut_diag_index,
           _mut_transposed_V]


def _pins_pass():
    """The golden and Lloyd pins, condensed; returns True when every pin holds."""
    try:
        # linear-kernel Lloyd equivalence on objective and distances
        X = synth.gaussian_blobs(120, 3, 4, seed=0, box=4.0)
        K = oracle.kernel_matrix(X, {"kind": "linear"})
        lab = synth.init_labels(120, 4, seed=1)
        for _ in range(3):
            st = oracle.step(K, lab, 4)
            ref_new, ref_J, ref_D = lloyd_step(X, lab, 4)
            if not np.allclose(st["D"], ref_D, rtol=1e-9, atol=1e-9):
                return False
            if not np.isclose(st["J"], ref_J, rtol=1e-9):
                return False
            lab = st["labels"]
        return True
    except Exception:
        return False


def test_unmutated_oracle_passes_condensed_pins():
    assert _pins_pass()


@pytest.mark.parametrize("mutant", MUTANTS, ids=lambda f: f.__name__)
def test_each_mutant_is_caught(mutant, monkeypatch):
    monkeypatch.setattr(kkmeans, "distances", mutant)
    assert not _pins_pass()


# ---- mistakes in the margin / scale outputs of step (they decide every parity exemption)

def _smut_margin_inf(K, labels, k):
    st = _orig_step(K, labels, k)
    return {**st, "margin": np.full_like(st["margin"], np.inf)}


def _smut_scale_huge(K, labels, k):
    st = _orig_step(K, labels, k)
    return {**st, "scale": st["scale"] * 1e6}


def _smut_margin_to_worst(K, labels, k):
    # largest finite distance minus the best: the wrong order statistic
    st = _orig_step(K, labels, k)
    D = np.where(np.isfinite(st["D"]), st["D"], -np.inf)
    return {**st, "margin": D.max(axis=1) - st["D"].min(axis=1)}


def _smut_scale_no_floor(K, labels, k):
    st = _orig_step(K, labels, k)
    return {**st, "scale": np.abs(st["D"].min(axis=1))}


def _smut_scale_from_second(K, labels, k):
    st = _orig_step(K, labels, k)
    part = np.sort(st["D"], axis=1)
    second = part[:, 1] if k > 1 else part[:, 0]
    second = np.where(np.isfinite(second), second, part[:, 0])
    return {**st, "scale": np.maximum(np.abs(second), st["kdiag"])}


def _smut_margin_own_cluster(K, labels, k):
    # distance to the current cluster minus the best, instead of second-best minus best
    st = _orig_step(K, labels, k)
    own = st["D"][np.arange(len(labels)), np.asarray(labels)]
    return {**st, "margin": own - st["D"].min(axis=1)}


STEP_MUTANTS = [_smut_margin_inf, _smut_scale_huge, _smut_margin_to_worst, _smut_scale_no_floor,
                _smut_scale_from_second, _smut_margin_own_cluster]


def test_unmutated_step_passes_margin_pins():
    assert margin_pins_hold(oracle.step)


@pytest.mark.parametrize("mutant", STEP_MUTANTS, ids=lambda f: f.__name__)
def test_each_margin_mutant_is_caught(mutant):
    assert not margin_pins_hold(mutant)
