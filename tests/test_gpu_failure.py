"""Failure detection, tested without a GPU fault.

Every wait inside the library's warp-specialized kernels is bounded: a wait that does
not see its phase within the limit raises the CTA's abort flag and an error word, every
role of the CTA leaves its loop, waits (bounded again) for its own copies in flight and
returns, and the host reports POPCORN_ERR_TIMEOUT.  These tests make such a wait run out
on purpose through the library's test hook: POPCORN_TEST_SYM_STALL_MS=<ms> makes the first
symmetric-stream launch of a fit (or the first tensor-core K stream of a batched fit) leave
one block's copies out (nothing ever arrives on that block's barrier) with every wait of the
launch bounded by <ms>; in the one-launch fit it makes one CTA leave before its first grid
barrier, so the others' bounded barrier waits run out.  Nothing faults or
hangs: the kernel returns, the call fails with the timeout status, and the next call on
the same context gives the reference result.  The other host-side failure paths (an
allocation the device cannot satisfy, a label out of range) are in test_gpu_parity.py.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


@pytest.mark.parametrize("sym_tile,storage", [(0, "fp32"), (1, "fp32"), (0, "bf16")],
                         ids=["sorted", "branch", "tensor_core"])
@pytest.mark.parametrize("check", [False, True], ids=["graph", "plain"])
def test_stream_wait_timeout_is_reported_and_the_context_survives(pc, monkeypatch, check, sym_tile, storage):
    """Every form of the symmetric stream: the sorted form (the automatic choice on an FP32
    K), the branch form (k <= 8 with a super-tile edge of 1) and the tensor-core form (a
    BF16 K: its producer leaves the block out, the MMA issuer's wait runs out)."""
    wl = synth.workload("rings", scale=0.1)              # n = 2,000: 136 blocks, one a CTA
    P = torch.from_numpy(wl.P).cuda()
    lab = torch.from_numpy(wl.init_labels).cuda()
    kw = dict(max_iter=6, check_convergence=check, history=True, k_pass="symmetric", sym_tile=sym_tile,
              k_storage=storage)
    ref = pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    assert ref["info"]["k_pass_used"] == 1
    # sums per row: sorted 12 registers, branch 4, tensor-core 16 TMEM columns
    assert ref["info"]["schedule"][3] == (16 if storage == "bf16" else 12 if sym_tile == 0 else 4)
    assert ref["info"]["sym_form"] == (3 if storage == "bf16" else 2 if sym_tile == 0 else 1)
    monkeypatch.setenv("POPCORN_TEST_SYM_STALL_MS", "200")
    t0 = time.perf_counter()
    with pytest.raises(pc.PopcornError) as ei:
        pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    assert ei.value.status == 4, str(ei.value)          # POPCORN_ERR_TIMEOUT
    assert "bounded wait" in str(ei.value)
    assert time.perf_counter() - t0 < 60
    monkeypatch.delenv("POPCORN_TEST_SYM_STALL_MS")
    torch.cuda.synchronize()                              # the context is intact
    again = pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    assert torch.equal(again["labels"], ref["labels"])
    assert again["objective"] == ref["objective"]
    assert again["info"]["J_history"] == ref["info"]["J_history"]


def test_stall_hook_is_inert_when_unset(pc):
    """Without the variable, or with the full-square pass (the hook touches the symmetric
    stream only), fits are the ordinary ones."""
    wl = synth.workload("blobs", scale=0.3)
    P = torch.from_numpy(wl.P).cuda()
    lab = torch.from_numpy(wl.init_labels).cuda()
    a = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=4, check_convergence=False, k_pass="full")
    b = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=4, check_convergence=False, k_pass="full")
    assert torch.equal(a["labels"], b["labels"]) and a["objective"] == b["objective"]
    assert np.isfinite(a["objective"])


def test_batched_tensor_core_stream_wait_timeout(pc, monkeypatch):
    """The batched tensor-core K stream (BF16 K): CTA 0 leaves one tile's copies out, the MMA
    issuer's bounded wait runs out, every role leaves, and the batch reports
    POPCORN_ERR_TIMEOUT; the context stays usable and the next batch is the ordinary one."""
    wls = synth.batched_instances(6, seed=5, n_lo=300, n_hi=1500)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]
    kw = dict(max_iter=4, check_convergence=False, k_storage="bf16")
    ref = pc.popcorn_fit_batched(insts, **kw)
    monkeypatch.setenv("POPCORN_TEST_SYM_STALL_MS", "200")
    t0 = time.perf_counter()
    with pytest.raises(pc.PopcornError) as ei:
        pc.popcorn_fit_batched(insts, **kw)
    assert ei.value.status == 4, str(ei.value)          # POPCORN_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60
    monkeypatch.delenv("POPCORN_TEST_SYM_STALL_MS")
    torch.cuda.synchronize()
    again = pc.popcorn_fit_batched(insts, **kw)
    for t in range(len(wls)):
        assert torch.equal(again["labels"][t], ref["labels"][t])
        assert again["objectives"][t] == ref["objectives"][t]


def test_grid_barrier_timeout_in_the_one_launch_fit(pc, monkeypatch):
    """The one-launch fit (K in L2, the automatic choice at this size): CTA 0 leaves before
    its first grid barrier, the other CTAs' bounded barrier waits run out, the fit reports
    POPCORN_ERR_TIMEOUT, and the next fit on the same context is the reference one."""
    wl = synth.workload("blobs")
    P = torch.from_numpy(wl.P).cuda()
    lab = torch.from_numpy(wl.init_labels).cuda()
    kw = dict(max_iter=10, check_convergence=False, history=True)
    ref = pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    assert ref["info"]["k_pass_used"] == 3
    monkeypatch.setenv("POPCORN_TEST_SYM_STALL_MS", "200")
    t0 = time.perf_counter()
    with pytest.raises(pc.PopcornError) as ei:
        pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    assert ei.value.status == 4, str(ei.value)          # POPCORN_ERR_TIMEOUT
    assert "grid barrier" in str(ei.value)
    assert time.perf_counter() - t0 < 60
    monkeypatch.delenv("POPCORN_TEST_SYM_STALL_MS")
    torch.cuda.synchronize()
    again = pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    assert torch.equal(again["labels"], ref["labels"])
    assert again["info"]["J_history"] == ref["info"]["J_history"]
