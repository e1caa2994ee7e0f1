"""popcorn_assign_step_noalloc against popcorn_assign_step, through the C ABI.

The no-allocation entry point is for callers that may not allocate device
memory (a host framework that owns all of it, a loop that forbids allocation
once running).  It must give the same answers as the allocating entry point,
call after call, while the shared static scratch keeps the previous call's
contents.  This file is collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes

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


def _noalloc_raw(pc, K, kd, labels, k):
    """Call the C entry point with caller-owned output buffers (allocated before the call)."""
    n = K.shape[0]
    new = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    counts = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    cnorm = torch.full((k,), -1.0, dtype=torch.float64, device="cuda")
    E = torch.full((n, k), -1.0, dtype=torch.float32, device="cuda")
    J = ctypes.c_double(0.0)
    ch = ctypes.c_int32(-1)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    allocs_before = pc._lib.popcorn_allocation_count()
    st = pc._lib.popcorn_assign_step_noalloc(
        ctypes.c_void_p(K.data_ptr()), K.stride(0), ctypes.c_void_p(kd.data_ptr()), n, k,
        ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(new.data_ptr()), ctypes.c_void_p(counts.data_ptr()),
        ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(cnorm.data_ptr()), ctypes.byref(J), ctypes.byref(ch),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert st == 0, pc._lib.popcorn_last_error_message()
    return {"labels": new, "counts": counts, "cnorm": cnorm, "E": E, "J": J.value, "changed": ch.value,
            "free_delta": free_before - free_after,
            "library_allocs": pc._lib.popcorn_allocation_count() - allocs_before}


def _case(n, d, k, seed, kern):
    P = synth.gaussian_blobs(n, d, min(k, 8), seed=seed, box=3.0)
    lab = synth.init_labels(n, k, seed=seed + 1)
    return P, lab, kern


CASES = [
    (3001, 5, 7, 11, {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 2.0}),
    (1500, 16, 3, 12, {"kind": "polynomial", "gamma": 1.0, "coef0": 1.0, "degree": 2, "sigma": 1.0}),
    (777, 4, 40, 13, {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 1.0}),
]


def test_noalloc_matches_allocating_step_on_consecutive_calls(pc):
    results = []
    for n, d, k, seed, kern in CASES:          # several calls in a row share the static scratch
        P, lab, kern = _case(n, d, k, seed, kern)
        K, kd = pc.popcorn_kernel_matrix(torch.from_numpy(P).cuda(), kern)
        labd = torch.from_numpy(lab).cuda()
        ref = pc.popcorn_assign_step(K, kd, labd, k, want_E=True)
        got = _noalloc_raw(pc, K, kd, labd, k)
        assert torch.equal(got["labels"], ref["labels"])
        assert torch.equal(got["counts"], ref["counts"])
        assert got["changed"] == ref["changed"]
        scale = float(K.abs().max())
        assert torch.allclose(got["E"], ref["E"], rtol=0, atol=1e-5 * scale)
        assert torch.allclose(got["cnorm"], ref["cnorm"], rtol=1e-5, atol=1e-6 * scale)
        assert rel_err(got["J"], ref["J"]) <= FP32_OBJ_REL
        # and both agree with the oracle's step (same parity rule as the other GPU tests)
        o = oracle.step(oracle.kernel_matrix(P, kern), lab, k)
        assert label_mismatches(got["labels"].cpu().numpy(), o)[0] == 0
        assert rel_err(got["J"], o["J"]) <= FP32_OBJ_REL
        results.append(got)
    # after the first call loaded the library's module, the calls allocate nothing; and no call,
    # the first included, takes a workspace block or a pinned host buffer from the library
    assert all(r["free_delta"] == 0 for r in results[1:])
    assert all(r["library_allocs"] == 0 for r in results)


def test_allocation_counter_sees_the_allocating_entry_point(pc):
    """The counter the test above relies on does move for the allocating step."""
    n, d, k, seed, kern = CASES[0]
    P, lab, kern = _case(n, d, k, seed, kern)
    K, kd = pc.popcorn_kernel_matrix(torch.from_numpy(P).cuda(), kern)
    before = pc._lib.popcorn_allocation_count()
    pc.popcorn_assign_step(K, kd, torch.from_numpy(lab).cuda(), k, want_E=True)
    torch.cuda.synchronize()
    assert pc._lib.popcorn_allocation_count() > before


def test_noalloc_repeat_call_is_identical(pc):
    n, d, k, seed, kern = CASES[0]
    P, lab, kern = _case(n, d, k, seed, kern)
    K, kd = pc.popcorn_kernel_matrix(torch.from_numpy(P).cuda(), kern)
    labd = torch.from_numpy(lab).cuda()
    a = _noalloc_raw(pc, K, kd, labd, k)
    b = _noalloc_raw(pc, K, kd, labd, k)
    assert torch.equal(a["labels"], b["labels"]) and torch.equal(a["counts"], b["counts"])
    assert torch.equal(a["E"], b["E"]) and a["J"] == b["J"]


def test_noalloc_rejects_sizes_beyond_its_scratch(pc):
    n, k = 200_000, 64                          # segment sums alone need > 32 MiB
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    lab = torch.zeros(16, dtype=torch.int32, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    st = pc._lib.popcorn_assign_step_noalloc(ptr, n, ptr, n, k, ctypes.c_void_p(lab.data_ptr()),
                                             ctypes.c_void_p(lab.data_ptr()), None, None, None, None, None,
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    msg = pc._lib.popcorn_last_error_message().decode()
    assert "scratch" in msg and str(pc.NOALLOC_SCRATCH_BYTES) in msg
