"""K stored in FP16 or BF16 (popcorn_options.k_storage): half the bytes per pass.

The build computes K in FP32 and rounds each entry once, so a pass is the
method run on round(K).  Bars from that arithmetic:
  * one pass against the FP64 oracle on the same rounded K: J to 1e-5, labels
    except near-ties below 2^-11 (FP16) / 2^-8 (BF16) of the row scale;
  * objective of the final labels against the FP64 oracle on the exact K:
    FP16 entries move by <= 2^-11 relative, BF16 by <= 2^-8 -- J moves by at
    most that times trace K / J; bars 1e-3 (FP16, Gaussian) and 1e-2 (BF16).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.parity import label_mismatches, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


def bf16_round64(x):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _rounded(K32, storage):
    if storage == "fp16":
        return K32.astype(np.float16).astype(np.float64)
    return bf16_round64(K32)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("storage,name,scale", [("fp16", "rings", 0.1), ("bf16", "rings", 0.1),
                                                ("bf16", "blobs", 0.5)])
def test_half_k_first_pass_matches_oracle_on_rounded_k(pc, storage, name, scale):
    wl = synth.workload(name, scale=scale)
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=1, check_convergence=False,
                       k_storage=storage, history=True)
    # the K the GPU rounds: its own FP32 build (checked against the oracle in the FP32 tests)
    K32, _ = pc.popcorn_kernel_matrix(_dev(wl.P), wl.kernel)
    Kr = _rounded(K32.cpu().numpy(), storage)
    st = oracle.step(Kr, wl.init_labels, wl.k)
    assert rel_err(r["info"]["J_history"][0], st["J"]) <= 1e-5
    rel = 2.0 ** -11 if storage == "fp16" else 2.0 ** -8
    assert label_mismatches(r["labels"].cpu().numpy(), st, rel=rel)[0] == 0


@pytest.mark.parametrize("storage,bar", [("fp16", 1e-3), ("bf16", 1e-2)])
def test_half_k_fit_objective_vs_exact(pc, storage, bar):
    wl = synth.workload("rings", scale=0.15)
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=wl.max_iter,
                       k_storage=storage)
    labels = r["labels"].cpu().numpy()
    J = oracle.objective(oracle.kernel_matrix(wl.P, wl.kernel), labels, wl.k)
    assert rel_err(r["objective"], J) <= bar, (r["objective"], J)


def test_half_k_ragged_and_host_buffers(pc):
    P = synth.gaussian_blobs(1001, 5, 3, seed=4, box=3.0)
    lab = synth.init_labels(1001, 7, seed=5)
    kern = {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 2.0}
    a = pc.popcorn_fit(P, 7, kern, lab, max_iter=20, k_storage="fp16")
    b = pc.popcorn_fit(_dev(P), 7, kern, _dev(lab), max_iter=20, k_storage="fp16")
    assert np.array_equal(a["labels"], b["labels"].cpu().numpy()) and a["objective"] == b["objective"]
