"""GPU parity of the one-launch fit (popcorn_fit on an FP32 K that sits in L2).

For n <= 6,144 and k <= 32 the automatic choice runs every pass of Alg. 2, and the final
objective pass, in one cooperative kernel with grid barriers between the phases of a pass
(k_pass_used = 3).  Its passes must be the oracle's steps (labels up to exempt near-ties, J
within the FP32 bar), its stopping rules those of the launched passes (fixed iterations,
convergence, the tolerance), and its outputs -- labels, objective, J / change histories,
E = K V^T, the loop state -- those of the same fit through the launched full-square passes
(k_pass = "full") up to FP32 summation order.  Runs are bit-identical.
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


def _gauss(s):
    return {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": s}


def _fit(pc, P, k, kern, lab, **kw):
    return pc.popcorn_fit(torch.from_numpy(P).cuda(), k, kern, torch.from_numpy(lab).cuda(), history=True, **kw)


def test_blobs_fit_is_the_oracle_fit(pc):
    """The blobs workload (n = 2,000, d = 16, k = 8, polynomial(1, 1, 2), 30 fixed passes):
    the one-launch fit follows the oracle's trajectory -- the same labels after every pass,
    J history and objective within the FP32 bar."""
    wl = synth.workload("blobs")
    r = _fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, max_iter=30, check_convergence=False)
    assert r["info"]["k_pass_used"] == 3
    Ko = oracle.kernel_matrix(wl.P, wl.kernel)
    o = oracle.fit(Ko, wl.k, wl.init_labels, 30, check_convergence=False)
    assert r["iterations"] == o["iterations"] == 30
    assert np.array_equal(r["labels"].cpu().numpy(), o["labels"])
    np.testing.assert_allclose(r["info"]["J_history"], o["J_history"], rtol=FP32_OBJ_REL)
    assert rel_err(r["objective"], o["objective"]) <= FP32_OBJ_REL


CASES = [
    # (n, d, k, kernel, seed)
    (2, 2, 1, _gauss(1.0), 1),            # the smallest problem: fewer rows than CTAs
    (97, 3, 3, _gauss(1.0), 2),
    (1030, 9, 8, _gauss(2.0), 3),         # n % 4 = 2 (scalar tail of every row)
    (2001, 5, 32, _gauss(1.5), 4),        # k at the bound
    (6144, 4, 10, _gauss(1.0), 5),        # n at the bound
    (3001, 6, 12, {"kind": "polynomial", "gamma": 0.5, "coef0": -1.0, "degree": 3, "sigma": 1.0}, 6),
]


@pytest.mark.parametrize("n,d,k,kern,seed", CASES)
def test_each_pass_is_the_oracle_step(pc, n, d, k, kern, seed):
    """Passes t = 1 and t = 3 of one-launch fits against the oracle's step from the labels
    the fit had after t - 1 passes (from the fit of t - 1 passes, itself one launch)."""
    P = synth.gaussian_blobs(n, d, k, seed=seed, box=3.0)
    lab = synth.init_labels(n, k, seed=seed + 100)
    Ko = oracle.kernel_matrix(P, kern)
    prev = lab
    for t in (1, 2, 3):
        r = _fit(pc, P, k, kern, lab, max_iter=t, check_convergence=False)
        assert r["info"]["k_pass_used"] == 3 and r["iterations"] == t
        if t != 2:
            st = oracle.step(Ko, prev, k)
            got = r["labels"].cpu().numpy()
            assert label_mismatches(got, st)[0] == 0
            assert rel_err(r["info"]["J_history"][t - 1], st["J"]) <= FP32_OBJ_REL
            assert rel_err(r["objective"], oracle.objective(Ko, got, k)) <= FP32_OBJ_REL
        prev = r["labels"].cpu().numpy()


@pytest.mark.parametrize("check,tol", [(True, 0.0), (True, 1e-3), (False, 0.0)])
def test_stopping_rules_match_the_launched_passes(pc, check, tol):
    """Rings at a quarter of its size (n = 5,000, k = 4): to convergence, with a tolerance,
    and for a fixed count, the one-launch fit stops where the launched passes stop, with the
    same labels and change history, J within the FP32 bar, and the same loop report."""
    wl = synth.workload("rings", scale=0.25)
    kw = dict(max_iter=100 if check else 25, check_convergence=check, tol=tol)
    a = _fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, **kw)
    b = _fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, k_pass="full", **kw)
    assert a["info"]["k_pass_used"] == 3 and b["info"]["k_pass_used"] == 2
    assert a["iterations"] == b["iterations"]
    assert a["info"]["converged"] == b["info"]["converged"]
    assert np.array_equal(a["labels"].cpu().numpy(), b["labels"].cpu().numpy())
    assert a["info"]["changed_history"] == b["info"]["changed_history"]
    np.testing.assert_allclose(a["info"]["J_history"], b["info"]["J_history"], rtol=FP32_OBJ_REL)
    assert rel_err(a["objective"], b["objective"]) <= FP32_OBJ_REL
    assert a["info"]["assign_launches"] == b["info"]["assign_launches"]
    assert a["info"]["reduce_launches"] == b["info"]["reduce_launches"]
    assert a["info"]["kernel_launches"] < b["info"]["kernel_launches"]


def test_zero_passes_and_the_E_report(pc):
    """max_iter = 0 evaluates J of the initial labels; E = K V^T of the labels the last pass
    started from matches the launched passes' report."""
    wl = synth.workload("blobs", scale=0.5)
    z = _fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, max_iter=0)
    Ko = oracle.kernel_matrix(wl.P, wl.kernel)
    assert z["iterations"] == 0 and z["info"]["k_pass_used"] == 3
    assert rel_err(z["objective"], oracle.objective(Ko, wl.init_labels, wl.k)) <= FP32_OBJ_REL
    E = [torch.empty((wl.n, wl.k), dtype=torch.float32, device="cuda") for _ in range(2)]
    a = _fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, max_iter=4, check_convergence=False, E_out=E[0])
    b = _fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, max_iter=4, check_convergence=False, E_out=E[1],
             k_pass="full")
    assert np.array_equal(a["labels"].cpu().numpy(), b["labels"].cpu().numpy())
    Ea, Eb = E[0].cpu().numpy(), E[1].cpu().numpy()
    assert np.max(np.abs(Ea - Eb)) <= 1e-5 * np.abs(Eb).max()


def test_runs_are_bit_identical(pc):
    """Integer counts by atomics (order-free), every floating-point sum in a fixed order."""
    wl = synth.workload("rings", scale=0.2)
    runs = [_fit(pc, wl.P, wl.k, wl.kernel, wl.init_labels, max_iter=60) for _ in range(3)]
    for r in runs[1:]:
        assert torch.equal(r["labels"], runs[0]["labels"])
        assert r["objective"] == runs[0]["objective"]
        assert r["info"]["J_history"] == runs[0]["info"]["J_history"]
        assert r["iterations"] == runs[0]["iterations"]
