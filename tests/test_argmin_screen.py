"""The FP32 screening rule of the argmin kernel, modelled on the CPU.

The kernel forms each distance D_ic = K_ii - 2 E_ic + ||c||^2 in FP32 (E_ic = S_ic / |L_c|
from an FP32 pair sum times an FP32 copy of 1/|L_c|, ||c||^2 rounded to FP32, one fused
multiply-add) and takes the FP32 argmin only when it beats every other cluster by more than
2B, B = 16 u (|K_ii| + max_c ||c||^2 + max_c |E_ic|), u = 2^-24; otherwise it decides the row in
FP64.  The claim: every row the screen passes has the FP64 argmin (lowest index on ties).
Here each FP32 step is one IEEE rounding of the exact value (numpy float32; the fused
multiply-add as one rounding of the FP64 value, exact for these operands), on rows built to
stress it: near-ties down to 1e-9 of the scale, |E| far above K_ii, negative entries (a
kernel that is not positive semi-definite), empty clusters, k = 1 and k = 256.
"""
import numpy as np
import pytest

U = 2.0 ** -24


def f32(x):
    return np.float32(x)


def screen_row(kd, S, invm, cnorm, counts):
    """(decided, cluster) of the FP32 screen for one row, and the FP64 argmin."""
    k = len(S)
    best64, b64 = np.inf, -1
    for c in range(k):
        if counts[c] == 0:
            continue
        E = float(np.float64(S[c]) * invm[c])
        D = (kd + cnorm[c]) - 2.0 * E
        if D < best64:
            best64, b64 = D, c
    kd32 = f32(kd)
    b1 = b2 = np.float32(np.inf)
    c1, emax, cmax = -1, np.float32(0), np.float32(0)
    for c in range(k):
        if counts[c] == 0:
            continue
        E32 = f32(np.float64(f32(S[c])) * np.float64(f32(invm[c])))
        t = f32(np.float64(kd32) + np.float64(f32(cnorm[c])))
        D32 = f32(-2.0 * np.float64(E32) + np.float64(t))          # one rounding: the FMA
        emax = max(emax, abs(E32))
        cmax = max(cmax, abs(f32(cnorm[c])))
        if D32 < b1:
            b2, b1, c1 = b1, D32, c
        elif D32 < b2:
            b2 = D32
    B = 16.0 * U * (abs(float(kd32)) + float(cmax) + float(emax))
    decided = float(b2) - float(b1) > 2.0 * B
    return decided, c1, b64


def _rows(rng, k, count, scale_e, negative, tie):
    for _ in range(count):
        counts = rng.integers(0, 5, size=k) * rng.integers(1, 40, size=k)
        counts[rng.integers(0, k)] = max(1, counts[rng.integers(0, k)])
        m = np.maximum(counts, 1).astype(np.float64)
        invm = 1.0 / m
        kd = float(rng.uniform(0.5, 2.0))
        E = rng.uniform(-1.0 if negative else 0.0, 1.0, size=k) * scale_e
        cnorm = rng.uniform(0.0, 1.0, size=k) * scale_e
        if tie is not None and k > 1:
            # two clusters within `tie` (relative) of each other, at the best value
            a, b = rng.choice(k, 2, replace=False)
            E[a] = E.max() + scale_e
            cnorm[a] = cnorm.min()
            E[b] = E[a] * (1.0 + tie * rng.uniform(-1, 1))
            cnorm[b] = cnorm[a]
            counts[a] = counts[b] = max(counts[a], 1)
        S = E * m          # the segment sum whose mean is E
        yield kd, S, invm, cnorm, counts


@pytest.mark.parametrize("k,scale_e,negative,tie", [
    (10, 1.0, False, None), (10, 1.0, False, 1e-6), (10, 1.0, False, 1e-9), (32, 50.0, False, 1e-5),
    (64, 1e4, True, 1e-7), (3, 1.0, True, 1e-3), (1, 1.0, False, None), (256, 10.0, True, 1e-6)])
def test_screen_never_disagrees_with_the_fp64_argmin(k, scale_e, negative, tie):
    rng = np.random.default_rng(k * 7 + int(scale_e))
    decided_rows = 0
    for kd, S, invm, cnorm, counts in _rows(rng, k, 400, scale_e, negative, tie):
        decided, c1, b64 = screen_row(kd, S, invm, cnorm, counts)
        if decided:
            decided_rows += 1
            assert c1 == b64
    if tie is None or tie >= 1e-5:
        assert decided_rows > 0          # the screen does decide most rows away from ties


def test_screen_defers_exact_ties_and_near_ties_to_fp64():
    """Two clusters at exactly the same FP64 distance, or within an FP32 rounding of it, are
    never decided by the screen (the FP64 path then takes the lower index)."""
    invm = np.array([0.25, 0.25, 0.5])
    counts = np.array([4, 4, 2])
    for d in (0.0, 1e-9, 1e-8):
        S = np.array([2.0, 2.0 * (1 + d), 0.1])
        decided, c1, b64 = screen_row(1.0, S, invm, np.array([0.3, 0.3, 0.9]), counts)
        assert not decided
