"""GPU parity of the tensor-core (tcgen05) K build and of fits that use it.

Bars (derived from the arithmetic):
  * small-integer points: every product and sum is exact in BF16 x BF16 -> FP32,
    so K must equal the oracle bit for bit in both BF16 and BF16X3 modes;
  * BF16 mode computes kappa of the BF16-rounded points (norms of the rounded
    rows): against the oracle on those rounded points, only FP32 accumulation
    error remains -> |dK| <= 2e-5 |K| + 2e-6 (Gaussian), rtol 2e-5 (polynomial);
  * BF16X3 carries ~16 significant bits of every coordinate: against the oracle
    on the raw FP32 points |dK| <= 2e-5 |K| + 2e-6 (Gaussian);
  * fits: BF16X3's objective for its final labels is within 1e-5 of the FP64
    oracle's objective of the same labels; BF16's is within 1e-5 of the oracle on
    the rounded points and within 2 * 2^-9 of the oracle on the raw points.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.parity import rel_err  # noqa: E402


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


def bf16_round(x):
    """Round float32 to the nearest bfloat16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


LINEAR = {"kind": "linear", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 1.0}
POLY2 = {"kind": "polynomial", "gamma": 1.0, "coef0": 1.0, "degree": 2, "sigma": 1.0}
POLY3 = {"kind": "polynomial", "gamma": 0.5, "coef0": 2.0, "degree": 3, "sigma": 1.0}


def gauss(s):
    return {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": s}


def test_bf16_round_helper():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 0.0, 65504.0], np.float32)
    r = bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0            # 1 + 2^-8 is a tie: to even
    assert r[2] == np.float32(1.0078125)          # above the tie: rounds up
    assert abs(r[3] - (-3.140625)) < 1e-7
    assert r[4] == 0.0


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("kern", [LINEAR, POLY2], ids=["linear", "poly2"])
def test_tc_exact_on_small_integers(pc, precision, kern):
    P = synth.small_integer_points(301, 8, seed=4)
    K, kd = pc.popcorn_kernel_matrix(_dev(P), kern, precision=precision)
    torch.cuda.synchronize()
    Ko = oracle.kernel_matrix(P, kern)
    np.testing.assert_array_equal(K.cpu().numpy().astype(np.float64), Ko)
    np.testing.assert_array_equal(kd.cpu().numpy(), np.diag(Ko).astype(np.float32))


@pytest.mark.parametrize("n,d", [(1, 3), (129, 1), (300, 70), (1000, 130), (517, 784)])
def test_tc_bf16_matches_oracle_on_rounded_points(pc, n, d):
    P = synth.sparse_images(n, d, 0.8, seed=n + d)
    Pr = bf16_round(P)
    for kern in (gauss(np.sqrt(d)), POLY2):
        K, kd = pc.popcorn_kernel_matrix(_dev(P), kern, precision="bf16")
        Kg = K.cpu().numpy().astype(np.float64)
        Ko = oracle.kernel_matrix(Pr, kern)
        if kern["kind"] == "gaussian":
            assert np.all(np.abs(Kg - Ko) <= 2e-5 * Ko + 2e-6)
            assert np.all(np.diag(Kg) == 1.0)
        else:
            np.testing.assert_allclose(Kg, Ko, rtol=2e-5, atol=1e-6 * np.abs(Ko).max())
        assert np.array_equal(Kg, Kg.T)


@pytest.mark.parametrize("n,d", [(129, 5), (700, 200), (517, 784)])
def test_tc_bf16x3_matches_oracle_on_raw_points(pc, n, d):
    P = synth.sparse_images(n, d, 0.8, seed=7 * n + d)
    kern = gauss(np.sqrt(d))
    K, _ = pc.popcorn_kernel_matrix(_dev(P), kern, precision="bf16x3")
    Kg = K.cpu().numpy().astype(np.float64)
    Ko = oracle.kernel_matrix(P, kern)
    err = np.abs(Kg - Ko)
    assert np.all(err <= 2e-5 * Ko + 2e-6), float(err.max())
    # off-diagonal tiles are stored from one value (exactly symmetric); inside a
    # diagonal tile K_ij and K_ji accumulate hi*lo and lo*hi at different depths
    assert np.max(np.abs(Kg - Kg.T)) <= 2e-6
    T = (n + 127) // 128
    for bi in range(T):
        for bj in range(bi + 1, T):
            blk = Kg[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128]
            assert np.array_equal(blk, Kg[bj * 128:(bj + 1) * 128, bi * 128:(bi + 1) * 128].T)


def test_tc_poly3_rings_bf16x3(pc):
    P = synth.gaussian_blobs(640, 16, 8, seed=3, box=2.0)
    K, _ = pc.popcorn_kernel_matrix(_dev(P), POLY3, precision="bf16x3")
    Ko = oracle.kernel_matrix(P, POLY3)
    np.testing.assert_allclose(K.cpu().numpy(), Ko, rtol=1e-4, atol=1e-4 * np.abs(Ko).max())


def test_tc_fit_objective_error_bf16x3(pc):
    wl = synth.workload("images", scale=0.02)          # n = 1400, d = 784, k = 10, Gaussian sigma 28
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=15,
                       precision="bf16x3", check_convergence=False, history=True)
    labels = r["labels"].cpu().numpy()
    J_true = oracle.objective(oracle.kernel_matrix(wl.P, wl.kernel), labels, wl.k)
    assert rel_err(r["objective"], J_true) <= 1e-5, (r["objective"], J_true)
    J = np.array(r["info"]["J_history"])
    assert np.all(np.diff(J) <= 1e-5 * np.abs(J[1:]))


def test_tc_fit_objective_error_bf16(pc):
    """BF16 mode clusters the BF16-rounded points: its objective matches the oracle on
    those points to 1e-5.  Against the raw points the rounding itself moves J: each
    coordinate moves by at most 2^-9 relative, so squared distances (and, in the
    near-linear regime of this workload, J) move by at most 2 * 2^-9 = 3.9e-3."""
    wl = synth.workload("images", scale=0.02)
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=15,
                       precision="bf16", check_convergence=False, history=True)
    labels = r["labels"].cpu().numpy()
    J_rounded = oracle.objective(oracle.kernel_matrix(bf16_round(wl.P), wl.kernel), labels, wl.k)
    assert rel_err(r["objective"], J_rounded) <= 1e-5, (r["objective"], J_rounded)
    J_true = oracle.objective(oracle.kernel_matrix(wl.P, wl.kernel), labels, wl.k)
    assert rel_err(r["objective"], J_true) <= 2 * 2.0 ** -9


def test_tc_full_size_images_sampled_rows(pc):
    """n = 70,000, d = 784 (19.6 GB K) with BF16X3: sampled rows against the oracle row by row."""
    wl = synth.workload("images")
    P = _dev(wl.P)
    K, kd = pc.popcorn_kernel_matrix(P, wl.kernel, precision="bf16x3")
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([rng.choice(wl.n, 24, replace=False), [0, 127, 128, wl.n - 1]]))
    Kr = oracle.kernel_matrix(wl.P[rows], wl.kernel, Q=wl.P)
    Kg = K[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    err = np.abs(Kg - Kr)
    assert np.all(err <= 2e-5 * Kr + 2e-6), float(err.max())
    # symmetry: the sampled rows equal the sampled columns (bit for bit outside diagonal tiles)
    Kc = K[:, torch.from_numpy(rows).cuda()].cpu().numpy().T.astype(np.float64)
    assert np.max(np.abs(Kg - Kc)) <= 2e-6
    assert float(kd.min()) == 1.0 and float(kd.max()) == 1.0
    del K
    torch.cuda.empty_cache()
