"""GPU parity of batched mode (popcorn_fit_batched): many instances in one graph.

Every instance must behave like an independent fit:
  * one pass from given labels: new labels equal the oracle's step except
    near-ties below 1e-6 of the row scale, and the objective of the new labels
    matches the oracle to 1e-6 (FP32);
  * whole fits: each instance's result equals a separate popcorn_fit of that
    instance (same method, same pass count) up to FP32 summation order, and
    converged labels are fixed points of the oracle's step;
  * instances that converge early stop while the others go on.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.parity import FP32_OBJ_REL, label_mismatches, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


def _batch(count=10, seed=3, n_lo=150, n_hi=1500):
    wls = synth.batched_instances(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]
    return wls, insts


def test_batched_one_pass_matches_oracle(pc):
    wls, insts = _batch()
    r = pc.popcorn_fit_batched(insts, max_iter=1, check_convergence=False)
    for t, w in enumerate(wls):
        Ko = oracle.kernel_matrix(w.P, w.kernel)
        st = oracle.step(Ko, w.init_labels, w.k)
        lab = r["labels"][t].cpu().numpy()
        assert r["iterations"][t] == 1
        assert label_mismatches(lab, st)[0] == 0, t
        assert rel_err(r["objectives"][t], oracle.objective(Ko, lab, w.k)) <= FP32_OBJ_REL, t


def test_batched_equals_separate_fits(pc):
    wls, insts = _batch(count=8, seed=5)
    r = pc.popcorn_fit_batched(insts, max_iter=40)
    for t, w in enumerate(wls):
        one = pc.popcorn_fit(insts[t]["P"], w.k, w.kernel, insts[t]["init_labels"], max_iter=40)
        lab = r["labels"][t].cpu().numpy()
        if np.array_equal(lab, one["labels"].cpu().numpy()):
            assert r["iterations"][t] == one["iterations"]
            assert rel_err(r["objectives"][t], one["objective"]) <= FP32_OBJ_REL
        Ko = oracle.kernel_matrix(w.P, w.kernel)
        assert rel_err(r["objectives"][t], oracle.objective(Ko, lab, w.k)) <= FP32_OBJ_REL
        if r["iterations"][t] < 40:                      # converged: a fixed point of the oracle's step
            assert label_mismatches(lab, oracle.step(Ko, lab, w.k))[0] == 0


def test_batched_uneven_convergence_and_zero_iterations(pc):
    wls, insts = _batch(count=6, seed=9)
    r = pc.popcorn_fit_batched(insts, max_iter=100)
    assert len(set(r["iterations"])) > 1                 # instances stop at different passes
    r0 = pc.popcorn_fit_batched(insts, max_iter=0)
    for t, w in enumerate(wls):
        assert r0["iterations"][t] == 0
        assert np.array_equal(r0["labels"][t].cpu().numpy(), w.init_labels)
        Ko = oracle.kernel_matrix(w.P, w.kernel)
        assert rel_err(r0["objectives"][t], oracle.objective(Ko, w.init_labels, w.k)) <= FP32_OBJ_REL


def test_batched_bf16x3_objective(pc):
    """bf16x3 keeps each coordinate to 2^-17 and drops lo*lo (2^-18), so B moves by <= 2^-16 of
    sum |p_l q_l|; the degree-2 polynomial doubles that in K (~3e-5) and J's cancellation
    (J well below trace K) amplifies it: bar 1e-4."""
    wls, insts = _batch(count=6, seed=11)
    r = pc.popcorn_fit_batched(insts, max_iter=10, precision="bf16x3", check_convergence=False)
    for t, w in enumerate(wls):
        Ko = oracle.kernel_matrix(w.P, w.kernel)
        lab = r["labels"][t].cpu().numpy()
        assert rel_err(r["objectives"][t], oracle.objective(Ko, lab, w.k)) <= 1e-4, t


def test_batched_rejects_bad_instance(pc):
    wls, insts = _batch(count=3, seed=1)
    insts[1] = dict(insts[1], k=10_000)
    with pytest.raises(pc.PopcornError) as ei:
        pc.popcorn_fit_batched(insts, max_iter=3)
    assert ei.value.status == 1 and "instance 1" in str(ei.value)


def test_batched_full_size_sampled(pc):
    """The 256-instance batch of the batched workload (n in [500, 8000]) in one graph, 29
    and 30 passes (deterministic runs: the 29-pass labels are the 30-pass run's labels
    before its last pass).  For sampled instances the oracle's step from the GPU's labels
    after pass 29 must give the GPU's labels after pass 30 (element by element up to
    exempt near-ties) and J of those labels; the reported objectives are J of the labels
    returned."""
    wls = synth.batched_instances(256, seed=0)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]
    r29 = pc.popcorn_fit_batched(insts, max_iter=29, check_convergence=False)
    l29 = [x.cpu().numpy() for x in r29["labels"]]
    r = pc.popcorn_fit_batched(insts, max_iter=30, check_convergence=False)
    for t in (0, 1, 77, 200, 255):
        w = wls[t]
        Ko = oracle.kernel_matrix(w.P, w.kernel)
        lab = r["labels"][t].cpu().numpy()
        assert r["iterations"][t] == 30 and r29["iterations"][t] == 29
        st = oracle.step(Ko, l29[t], w.k)
        assert rel_err(r29["objectives"][t], st["J"]) <= FP32_OBJ_REL, t
        assert label_mismatches(lab, st)[0] == 0, t
        assert rel_err(r["objectives"][t], oracle.objective(Ko, lab, w.k)) <= FP32_OBJ_REL, t


# ---------------------------------------------------------------- half-precision K
# k_storage "fp16" / "bf16": every instance's square rounded once (after the FP32 or tensor-
# core build) into 32 KB tiles read by the tensor-core stream (MMAs of each tile against
# one-hot label operands, FP32 sums in TMEM).  The method then runs on the rounded K: one
# pass must be the oracle's step on the oracle's K rounded the same way (through FP32),
# labels up to near-ties within the storage type's relative rounding.


def _rounded_k(P, kern, storage):
    K32 = oracle.kernel_matrix(P, kern).astype(np.float32)
    if storage == "fp16":
        return K32.astype(np.float16).astype(np.float64)
    u = K32.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def _gauss_only(insts, wls):
    keep = [t for t, w in enumerate(wls) if w.kernel["kind"] == "gaussian"]   # |K| <= 1: FP16-safe
    return [insts[t] for t in keep], [wls[t] for t in keep]


@pytest.mark.parametrize("storage,precision", [("bf16", "fp32"), ("fp16", "fp32"), ("bf16", "bf16")])
def test_batched_half_k_one_pass_matches_oracle_on_rounded_k(pc, storage, precision):
    wls, insts = _batch(count=12, seed=13)
    if storage == "fp16":
        insts, wls = _gauss_only(insts, wls)
    assert len(wls) >= 4
    r = pc.popcorn_fit_batched(insts, max_iter=1, check_convergence=False, k_storage=storage, precision=precision)
    rel = 2.0 ** -10 if storage == "fp16" else 2.0 ** -7
    for t, w in enumerate(wls):
        P = w.P
        if precision == "bf16":   # the BF16 build: K of the rounded points
            P = torch.from_numpy(w.P).to(torch.bfloat16).to(torch.float64).numpy()
        Kr = _rounded_k(P, w.kernel, storage)
        st = oracle.step(Kr, w.init_labels, w.k)
        lab = r["labels"][t].cpu().numpy()
        assert r["iterations"][t] == 1
        assert label_mismatches(lab, st, rel=rel)[0] == 0, t
        assert rel_err(r["objectives"][t], oracle.objective(Kr, lab, w.k)) <= 1e-5, t


def test_batched_half_k_whole_fits_and_info(pc):
    """Whole fits with convergence checking: every instance stops at a fixed point of the
    oracle's step on its rounded K (up to near-ties), instances stop at different passes,
    and the reported objective is J of the returned labels on the rounded K; the schedule
    reports the ring depth and the widest accumulator (k rounded up to 16)."""
    wls, insts = _batch(count=8, seed=15)
    r = pc.popcorn_fit_batched(insts, max_iter=60, k_storage="bf16")
    assert r["info"]["schedule"][3] == max((w.k + 15) // 16 * 16 for w in wls)
    assert r["info"]["schedule"][1] >= 2
    assert len(set(r["iterations"])) > 1
    for t, w in enumerate(wls):
        Kr = _rounded_k(w.P, w.kernel, "bf16")
        lab = r["labels"][t].cpu().numpy()
        assert rel_err(r["objectives"][t], oracle.objective(Kr, lab, w.k)) <= 1e-5, t
        if r["iterations"][t] < 60:
            assert label_mismatches(lab, oracle.step(Kr, lab, w.k), rel=2.0 ** -7)[0] == 0, t


def test_batched_half_k_full_size_sampled(pc):
    """The 256-instance batch of the batched workload with a BF16 K: 29 and 30 passes; for
    sampled instances the oracle's step (rounded K) from the GPU's labels after pass 29 gives
    the GPU's labels after pass 30 (up to exempt near-ties) and J of those labels."""
    wls = synth.batched_instances(256, seed=0)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]
    r29 = pc.popcorn_fit_batched(insts, max_iter=29, check_convergence=False, k_storage="bf16")
    l29 = [x.cpu().numpy() for x in r29["labels"]]
    r = pc.popcorn_fit_batched(insts, max_iter=30, check_convergence=False, k_storage="bf16")
    for t in (0, 1, 77, 200, 255):
        w = wls[t]
        Kr = _rounded_k(w.P, w.kernel, "bf16")
        lab = r["labels"][t].cpu().numpy()
        st = oracle.step(Kr, l29[t], w.k)
        assert rel_err(r29["objectives"][t], st["J"]) <= 1e-5, t
        assert label_mismatches(lab, st, rel=2.0 ** -7)[0] == 0, t
        assert rel_err(r["objectives"][t], oracle.objective(Kr, lab, w.k)) <= 1e-5, t


def test_batched_half_k_tiny_and_ragged_instances(pc):
    """Instances smaller than one 128-block, exactly one block, one point past it, and k from
    1 to n - 1 and up to 200 (N = 16 to 208 accumulator columns) in one half-K batch: one pass
    each against the oracle's step on the rounded K."""
    rng = np.random.default_rng(41)
    # k up to 200: N = 208 accumulator columns, two ring stages of 32 KB + 52 KB, 512 TMEM columns
    shapes = [(2, 1), (5, 4), (40, 39), (127, 20), (128, 64), (129, 3), (300, 1), (700, 50), (900, 130),
              (1500, 200)]
    wls, insts = [], []
    for t, (n, k) in enumerate(shapes):
        P = rng.normal(size=(n, 6)).astype(np.float32) * 2.0
        lab = synth.init_labels(n, k, seed=60 + t)
        kern = {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 3.0}
        wls.append((P, lab, k, kern))
        insts.append({"P": torch.from_numpy(P).cuda(), "k": k, "kernel": kern,
                      "init_labels": torch.from_numpy(lab).cuda()})
    for storage in ("fp16", "bf16"):
        r = pc.popcorn_fit_batched(insts, max_iter=1, check_convergence=False, k_storage=storage)
        rel = 2.0 ** -10 if storage == "fp16" else 2.0 ** -7
        for t, (P, lab, k, kern) in enumerate(wls):
            Kr = _rounded_k(P, kern, storage)
            st = oracle.step(Kr, lab, k)
            got = r["labels"][t].cpu().numpy()
            assert label_mismatches(got, st, rel=rel)[0] == 0, (storage, t)
            assert rel_err(r["objectives"][t], oracle.objective(Kr, got, k)) <= 1e-5, (storage, t)
