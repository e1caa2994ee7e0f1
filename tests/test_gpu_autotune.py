"""GPU tests of the autotuner (options.autotune = 1).

The tuner only changes the schedule -- K-stream unit length, warps and blocks
per SM (batched mode); row blocks per tile and units per SM (recompute path) --
so a tuned fit must give the untuned fit's result up to FP32 summation order:
labels equal except near-ties, objective within the FP32 bar (or the BF16/FP8
bar on the recompute path).  A second call with the same workload signature
must reuse the cached schedule without timing anything.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.parity import FP32_OBJ_REL, rel_err  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


def _batch(count=12, seed=11):
    wls = synth.batched_instances(count, seed=seed, n_lo=300, n_hi=3000)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]
    return wls, insts


def test_batched_autotune_then_cache_hit(pc):
    pc.popcorn_autotune_clear()
    wls, insts = _batch()
    base = pc.popcorn_fit_batched(insts, max_iter=8, check_convergence=False)
    t1 = pc.popcorn_fit_batched(insts, max_iter=8, check_convergence=False, autotune=True)
    i1 = t1["info"]
    assert i1["tune_cache_hit"] == 0 and i1["tune_candidates"] >= 4
    seglen, warps, per_sm, _ = i1["schedule"]
    assert seglen in (2048, 4096, 8192, 16384) and warps in (4, 8, 16) and per_sm in (1, 2)
    assert pc.popcorn_autotune_entries() == 1
    t2 = pc.popcorn_fit_batched(insts, max_iter=8, check_convergence=False, autotune=True)
    assert t2["info"]["tune_cache_hit"] == 1 and t2["info"]["tune_candidates"] == 0
    assert t2["info"]["schedule"] == i1["schedule"]
    for t, w in enumerate(wls):
        Ko = oracle.kernel_matrix(w.P, w.kernel)
        for r in (t1, t2):
            lab = r["labels"][t].cpu().numpy()
            # the tuned schedule changes summation order only
            assert rel_err(r["objectives"][t], oracle.objective(Ko, lab, w.k)) <= FP32_OBJ_REL, t
            same = np.mean(lab == base["labels"][t].cpu().numpy())
            assert same >= 0.99, (t, same)
        assert t1["iterations"][t] == base["iterations"][t] == 8


def test_batched_untuned_reports_heuristic_schedule(pc):
    _, insts = _batch(count=4, seed=2)
    r = pc.popcorn_fit_batched(insts, max_iter=2)
    assert r["info"]["tune_candidates"] == 0 and r["info"]["tune_cache_hit"] == 0
    assert r["info"]["schedule"][0] == 8192 and r["info"]["schedule"][1] >= 1


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_recompute_autotune_matches_untuned(pc, precision):
    pc.popcorn_autotune_clear()
    wl = synth.workload("mixture", scale=0.04)          # n = 8000, d = 128, k = 100
    P = torch.from_numpy(wl.P).cuda()
    L0 = torch.from_numpy(wl.init_labels).cuda()
    base = pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=3, precision=precision, store_k=False,
                          check_convergence=False)
    r = pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=3, precision=precision, store_k=False,
                       check_convergence=False, autotune=True)
    info = r["info"]
    assert info["tune_candidates"] >= 2 and info["tune_cache_hit"] == 0
    rbp, nseg, upsm, _ = info["schedule"]
    assert rbp in (1, 2) and nseg >= 1 and upsm in (8, 16, 32)
    assert rel_err(r["objective"], base["objective"]) <= 1e-4
    same = np.mean(r["labels"].cpu().numpy() == base["labels"].cpu().numpy())
    assert same >= 0.99
    r2 = pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=3, precision=precision, store_k=False,
                        check_convergence=False, autotune=True)
    assert r2["info"]["tune_cache_hit"] == 1 and r2["info"]["schedule"][:3] == [rbp, nseg, upsm]


def test_tuned_schedule_persists_across_processes(pc, tmp_path):
    """A process with POPCORN_TUNE_CACHE set appends its tuned schedule; the next
    process reads it and skips the timing."""
    path = tmp_path / "tune.txt"
    code = ("import torch, synth, paper_2501_05587_gb300 as pc\n"
            "wls = synth.batched_instances(6, seed=4, n_lo=300, n_hi=2000)\n"
            "ins = [{'P': torch.from_numpy(w.P).cuda(), 'k': w.k, 'kernel': w.kernel,"
            " 'init_labels': torch.from_numpy(w.init_labels).cuda()} for w in wls]\n"
            "r = pc.popcorn_fit_batched(ins, max_iter=2, autotune=True)\n"
            "print(r['info']['tune_cache_hit'], r['info']['tune_candidates'])\n")
    env = dict(os.environ, POPCORN_TUNE_CACHE=str(path))
    outs = []
    for _ in range(2):
        p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        assert p.returncode == 0, p.stderr
        outs.append(p.stdout.split())
    assert outs[0][0] == "0" and int(outs[0][1]) > 0
    assert outs[1] == ["1", "0"]
    assert path.read_text().count("\n") == 1
