"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Sizes span several 128-wide tiles and a ragged tail (n not a multiple of 4,
128 or the row-segment length).  Bars (written in each test):
  * K (FP32 build): |K_gpu - K| <= 2e-6 |K| + 1e-6 max|K| (linear / polynomial),
    exact for small-integer points; Gaussian |K_gpu - K| <= 1e-6.
  * E = K V^T: within 1e-5 of the row scale.
  * labels: equal except oracle margins below 1e-6 * scale (spec rule).
  * objective: relative error <= 1e-6 (FP32 path).
"""
import math

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


def _dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def _poly(g=1.0, c=1.0, r=2):
    return {"kind": "polynomial", "gamma": g, "coef0": c, "degree": r, "sigma": 1.0}


def _gauss(s):
    return {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": s}


LINEAR = {"kind": "linear", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 1.0}


# ------------------------------------------------------------------ K build

@pytest.mark.parametrize("n,d", [(1, 3), (5, 1), (127, 4), (333, 5), (517, 16), (1030, 9)])
@pytest.mark.parametrize("kern", [LINEAR, _poly(1.0, 1.0, 2), _poly(0.5, 2.0, 3), _gauss(1.5)],
                         ids=["linear", "poly2", "poly3", "gauss"])
def test_kernel_matrix_fp32(pc, n, d, kern):
    P = synth.gaussian_blobs(n, d, 3, seed=n + d, box=2.0)
    K, kd = pc.popcorn_kernel_matrix(_dev(P), kern)
    torch.cuda.synchronize()
    Kg = K.cpu().numpy().astype(np.float64)
    Ko = oracle.kernel_matrix(P, kern)
    if kern["kind"] == "gaussian":
        assert np.max(np.abs(Kg - Ko)) <= 1e-6
        assert np.all(np.diag(Kg) == 1.0)
    else:
        tol = 2e-6 * np.abs(Ko) + 1e-6 * np.abs(Ko).max()
        assert np.all(np.abs(Kg - Ko) <= tol)
    assert np.array_equal(Kg, Kg.T)
    np.testing.assert_array_equal(kd.cpu().numpy(), np.diag(K.cpu().numpy()))


@pytest.mark.parametrize("kern", [LINEAR, _poly(1.0, 1.0, 2), _poly(1.0, 3.0, 3)], ids=["linear", "poly2", "poly3"])
def test_kernel_matrix_exact_on_small_integers(pc, kern):
    P = synth.small_integer_points(301, 8, seed=3)
    K, _ = pc.popcorn_kernel_matrix(_dev(P), kern)
    Ko = oracle.kernel_matrix(P, kern)
    assert np.abs(Ko).max() < 2 ** 24
    np.testing.assert_array_equal(K.cpu().numpy().astype(np.float64), Ko)


def test_kernel_matrix_strided_points(pc):
    P = synth.gaussian_blobs(200, 6, 2, seed=1)
    big = torch.zeros((200, 11), dtype=torch.float32, device="cuda")
    big[:, :6] = _dev(P)
    K, _ = pc.popcorn_kernel_matrix(big[:, :6], _poly())
    np.testing.assert_allclose(K.cpu().numpy(), oracle.kernel_matrix(P, _poly()), rtol=2e-6, atol=1e-4)


# ------------------------------------------------------------------ one pass, teacher-forced

def _step_case(pc, P, kern, labels, k):
    Pd = _dev(P)
    K, kd = pc.popcorn_kernel_matrix(Pd, kern)
    g = pc.popcorn_assign_step(K, kd, _dev(labels), k, want_E=True)
    torch.cuda.synchronize()
    Ko = oracle.kernel_matrix(P, kern)
    o = oracle.step(Ko, labels, k)
    return g, o, Ko


def _check_step(g, o, Ko, obj_rel=FP32_OBJ_REL):
    n, k = o["E"].shape
    E = g["E"].cpu().numpy().astype(np.float64)
    row_scale = np.abs(Ko).max(axis=1)[:, None]
    assert np.all(np.abs(E - o["E"]) <= 1e-5 * row_scale + 1e-30)
    cn = g["cnorm"].cpu().numpy()
    nonempty = o["counts"] > 0
    np.testing.assert_allclose(cn[nonempty], o["cnorm"][nonempty], rtol=1e-5, atol=1e-6 * np.abs(Ko).max())
    assert rel_err(g["J"], o["J"]) <= obj_rel, (g["J"], o["J"])
    bad, _ = label_mismatches(g["labels"].cpu().numpy(), o)
    assert bad == 0
    new = g["labels"].cpu().numpy()
    np.testing.assert_array_equal(g["counts"].cpu().numpy(), np.bincount(new, minlength=k))
    assert g["changed"] == int((new != o["labels_in"]).sum())


@pytest.mark.parametrize("n,k", [(2, 1), (3, 2), (129, 3), (1001, 7), (4099, 16), (2500, 64), (700, 256)])
def test_assign_step_matches_oracle(pc, n, k):
    P = synth.gaussian_blobs(n, 5, max(1, min(k, 8)), seed=n, box=3.0)
    kern = _gauss(2.0)
    lab = synth.init_labels(n, k, seed=n + 1)
    g, o, Ko = _step_case(pc, P, kern, lab, k)
    o["labels_in"] = lab
    _check_step(g, o, Ko)


@pytest.mark.parametrize("kern", [LINEAR, _poly(), _gauss(0.5)], ids=["linear", "poly", "gauss"])
def test_assign_step_kernels(pc, kern):
    P = synth.rings(1500, seed=2, d_pad=8) if kern["kind"] == "gaussian" else \
        synth.gaussian_blobs(1500, 16, 8, seed=2)
    lab = synth.init_labels(1500, 8, seed=3)
    g, o, Ko = _step_case(pc, P, kern, lab, 8)
    o["labels_in"] = lab
    _check_step(g, o, Ko)


def test_assign_step_empty_cluster_and_in_place(pc):
    n, k = 600, 5
    P = synth.gaussian_blobs(n, 3, 4, seed=5)
    lab = synth.init_labels(n, k, seed=6)
    lab[lab == 2] = 4                                      # cluster 2 empty
    Pd = _dev(P)
    K, kd = pc.popcorn_kernel_matrix(Pd, _poly())
    labd = _dev(lab)
    g = pc.popcorn_assign_step(K, kd, labd, k, want_E=True)
    o = oracle.step(oracle.kernel_matrix(P, _poly()), lab, k)
    new = g["labels"].cpu().numpy()
    assert not np.any(new == 2)
    assert np.all(g["E"].cpu().numpy()[:, 2] == 0)
    assert g["cnorm"].cpu().numpy()[2] == 0
    assert label_mismatches(new, o)[0] == 0


def test_assign_step_rejects_bad_labels(pc):
    P = synth.gaussian_blobs(100, 3, 2, seed=1)
    K, kd = pc.popcorn_kernel_matrix(_dev(P), LINEAR)
    lab = synth.init_labels(100, 3, seed=1)
    lab[17] = 3
    with pytest.raises(pc.PopcornError) as ei:
        pc.popcorn_assign_step(K, kd, _dev(lab), 3)
    assert ei.value.status == 1
    # the context stays usable
    lab[17] = 0
    pc.popcorn_assign_step(K, kd, _dev(lab), 3)


# ------------------------------------------------------------------ whole fits

def _fit_parity(pc, wl, max_iter=None, check=None, host=False):
    """popcorn_fit against the oracle's loop.

    When the two trajectories agree label for label, the objective history and
    change counts must agree.  When they split (an exempt near-tie resolved the
    other way), parity is checked per pass: the GPU's labels after t passes
    (popcorn_fit with max_iter = t, a prefix of the same deterministic run) are
    fed to the oracle, whose step must reproduce the GPU's J_t and labels
    after pass t + 1 up to exempt near-ties.
    """
    max_iter = wl.max_iter if max_iter is None else max_iter
    check = wl.check_convergence if check is None else check
    if host:
        P, lab = wl.P, wl.init_labels
    else:
        P, lab = _dev(wl.P), _dev(wl.init_labels)
    r = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=max_iter, check_convergence=check, history=True)
    torch.cuda.synchronize()
    Ko = oracle.kernel_matrix(wl.P, wl.kernel)
    o = oracle.fit(Ko, wl.k, wl.init_labels, max_iter, check_convergence=check)
    labels = r["labels"] if host else r["labels"].cpu().numpy()
    same = (r["iterations"] == o["iterations"] and r["info"]["changed_history"] == o["changed_history"]
            and np.array_equal(labels, o["labels"])
            and np.allclose(r["info"]["J_history"], o["J_history"], rtol=FP32_OBJ_REL, atol=0))
    if not same:
        prev = wl.init_labels
        for t in range(r["iterations"]):
            nxt = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=t + 1, check_convergence=False)["labels"]
            nxt = nxt if host else nxt.cpu().numpy()
            st = oracle.step(Ko, prev, wl.k)
            assert rel_err(r["info"]["J_history"][t], st["J"]) <= FP32_OBJ_REL, t
            assert label_mismatches(nxt, st)[0] == 0, t
            assert r["info"]["changed_history"][t] == int((nxt != prev).sum()), t
            prev = nxt
        assert np.array_equal(prev, labels)
    st = oracle.step(Ko, labels, wl.k)
    assert rel_err(r["objective"], st["J"]) <= FP32_OBJ_REL
    if check and r["info"]["converged"]:
        assert label_mismatches(labels, st)[0] == 0
    return r, o, same


@pytest.mark.parametrize("name,scale", [("blobs", 1.0), ("rings", 0.15), ("images", 0.02)])
def test_fit_matches_oracle(pc, name, scale):
    wl = synth.workload(name, scale=scale)
    max_iter = min(wl.max_iter, 30)
    r, o, _ = _fit_parity(pc, wl, max_iter=max_iter)
    J = np.array(r["info"]["J_history"])
    assert np.all(np.diff(J) <= 1e-6 * np.abs(J[1:]))    # non-increasing (FP32 tolerance)


def test_fit_host_buffers_equal_device_buffers(pc):
    wl = synth.workload("rings", scale=0.1)
    rd = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=40, history=True)
    rh = pc.popcorn_fit(wl.P, wl.k, wl.kernel, wl.init_labels, max_iter=40, history=True)
    assert np.array_equal(rd["labels"].cpu().numpy(), rh["labels"])
    assert rd["objective"] == rh["objective"]
    assert rd["iterations"] == rh["iterations"]
    assert rh["info"]["h2d_bytes"] == wl.P.nbytes + wl.init_labels.nbytes
    assert rh["info"]["d2h_bytes"] >= wl.init_labels.nbytes


def test_fit_stopping_rules(pc):
    wl = synth.workload("blobs", scale=0.2)
    r0 = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=0)
    assert r0["iterations"] == 0
    assert np.array_equal(r0["labels"].cpu().numpy(), wl.init_labels)
    Ko = oracle.kernel_matrix(wl.P, wl.kernel)
    assert rel_err(r0["objective"], oracle.objective(Ko, wl.init_labels, wl.k)) <= FP32_OBJ_REL
    rc = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=100, history=True)
    oc = oracle.fit(Ko, wl.k, wl.init_labels, 100)
    assert rc["info"]["converged"] == 1 and oc["converged"]
    assert rc["iterations"] == oc["iterations"]
    rf = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=7, check_convergence=False)
    assert rf["iterations"] == 7
    rt = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=100, tol=1e-2, history=True)
    ot = oracle.fit(Ko, wl.k, wl.init_labels, 100, tol=1e-2)
    assert rt["iterations"] == ot["iterations"]


@pytest.mark.parametrize("k_pass", ["full", "auto"])
def test_fit_repeatable_and_timing_info(pc, k_pass):
    """Per-kernel timing of the launched passes ("full"), and of the one-launch fit that the
    automatic choice takes at this size (n = 2,000: its passes are inside one kernel, so only
    the build and the loop are timed)."""
    wl = synth.workload("rings", scale=0.1)
    P, lab = _dev(wl.P), _dev(wl.init_labels)
    a = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=50, timing=True, k_pass=k_pass)
    b = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=50, k_pass=k_pass)
    assert torch.equal(a["labels"], b["labels"]) and a["objective"] == b["objective"]
    inf = a["info"]
    assert inf["reduce_launches"] >= a["iterations"] and inf["assign_launches"] == a["iterations"]
    assert inf["kbuild_ms"] > 0 and inf["loop_ms"] > 0
    if k_pass == "full":
        assert inf["k_pass_used"] == 2 and inf["reduce_ms"] > 0 and inf["loop_ms"] >= inf["reduce_ms"]
    else:
        assert inf["k_pass_used"] == 3 and inf["reduce_ms"] == 0


# ------------------------------------------------------------------ full-size checks

def test_full_size_rings_sampled(pc):
    """n = 20000 rings through popcorn_kernel_matrix (full-square FP32 K) and
    popcorn_assign_step (the full-square pass): sampled rows of K and E against the
    oracle row by row, J against the identity trace K - sum |L_c| ||c_c||^2.  The
    symmetric pass that popcorn_fit runs on this workload is checked against the
    oracle's step at this size in test_gpu_sym.py."""
    wl = synth.workload("rings")
    P = _dev(wl.P)
    K, kd = pc.popcorn_kernel_matrix(P, wl.kernel)
    g = pc.popcorn_assign_step(K, kd, _dev(wl.init_labels), wl.k, want_E=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.choice(wl.n, 48, replace=False), [0, wl.n - 1]]))
    Kr = oracle.kernel_matrix(wl.P[rows], wl.kernel, Q=wl.P)
    Kg = K[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Kg - Kr)) <= 1e-6
    lab = wl.init_labels.astype(np.int64)
    counts = np.bincount(lab, minlength=wl.k)
    onehot = np.zeros((wl.n, wl.k))
    onehot[np.arange(wl.n), lab] = 1.0 / counts[lab]
    Eo = Kr @ onehot
    Eg = g["E"][torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Eg - Eo)) <= 1e-5 * max(1.0, np.abs(Eo).max())
    # identity: J = sum_i K_ii - sum_c |L_c| ||c_c||^2
    cn = g["cnorm"].cpu().numpy()
    J_id = float(kd.double().sum().item()) - float((counts * cn).sum())
    assert rel_err(g["J"], J_id) <= 1e-9


def test_full_size_rings_fit_monotone(pc):
    wl = synth.workload("rings")
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=wl.max_iter, history=True)
    J = np.array(r["info"]["J_history"])
    assert len(J) == r["iterations"] >= 1
    assert np.all(np.diff(J) <= 1e-6 * np.abs(J[1:]))
    if r["info"]["converged"]:
        assert r["info"]["changed_history"][-1] == 0
        assert rel_err(r["objective"], J[-1]) <= 1e-12


def test_fit_reports_nomem_and_stays_usable(pc):
    """A stored K that cannot fit in device memory (n = 400,000: 320 GB even as the
    packed upper triangle) is refused with POPCORN_ERR_NOMEM before any kernel runs,
    nothing is leaked, and the next call works."""
    n = 400_000
    P = np.zeros((n, 1), dtype=np.float32)
    P[:, 0] = np.linspace(-1.0, 1.0, n, dtype=np.float32)
    lab = (np.arange(n) % 4).astype(np.int32)
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(pc.PopcornError) as ei:
        pc.popcorn_fit(P, 4, _gauss(1.0), lab, max_iter=2)
    assert ei.value.status == 2, str(ei.value)
    assert "kernel matrix" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    wl = synth.workload("blobs", scale=0.1)
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=3)
    assert r["iterations"] >= 1


@pytest.mark.parametrize("name,scale,k_pass", [("blobs", 1.0, "full"), ("rings", 0.2, "symmetric"),
                                               ("rings", 0.2, "full"), ("images", 0.03, "full")])
def test_fixed_iteration_graph_equals_plain_launches(pc, name, scale, k_pass):
    """A fixed-iteration fit without per-kernel events runs all its passes and the objective
    pass as one CUDA graph.  The kernels, their arguments and their order are those of the
    plainly launched fit (timing = 1), and every reduction order is fixed, so labels,
    objective and the J / change histories are bit-identical; phase timing reports the
    graph's time as loop_ms."""
    wl = synth.workload(name, scale=scale)
    P, lab = _dev(wl.P), _dev(wl.init_labels)
    kw = dict(max_iter=12, check_convergence=False, history=True, k_pass=k_pass)
    g = pc.popcorn_fit(P, wl.k, wl.kernel, lab, **kw)
    h = pc.popcorn_fit(P, wl.k, wl.kernel, lab, timing="phases", **kw)
    p = pc.popcorn_fit(P, wl.k, wl.kernel, lab, timing=True, **kw)
    for r in (g, h):
        assert torch.equal(r["labels"], p["labels"])
        assert r["objective"] == p["objective"]
        assert r["info"]["J_history"] == p["info"]["J_history"]
        assert r["info"]["changed_history"] == p["info"]["changed_history"]
        assert r["iterations"] == p["iterations"] == 12
        assert r["info"]["kernel_launches"] == p["info"]["kernel_launches"]
    assert h["info"]["loop_ms"] > 0 and h["info"]["reduce_ms"] == 0 and h["info"]["kbuild_ms"] > 0
    assert p["info"]["reduce_ms"] > 0


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "bf16"])
@pytest.mark.parametrize("kern", [LINEAR, _gauss(3.0)], ids=["linear", "gauss"])
def test_kernel_matrix_schedules_agree(pc, precision, kern):
    """The full tile schedule (every tile formed, the GEMM form) and the symmetric one (tiles
    on and above the diagonal stored with their transposes, the SYRK form) build the same K:
    bit for bit in FP32 (the same products added in the same order), to accumulation-order
    rounding in the tensor-core forms.  The tuned schedule is one of the two; FP32 against
    the oracle as in test_kernel_matrix_fp32."""
    n, d = 700, 37                                   # 6 tiles a side, ragged; d not a multiple of 64
    P = synth.gaussian_blobs(n, d, 3, seed=17, box=2.0)
    Pd = _dev(P)
    Ks, ds = pc.popcorn_kernel_matrix(Pd, kern, precision, schedule="symmetric")
    Kf, df = pc.popcorn_kernel_matrix(Pd, kern, precision, schedule="full")
    Kt, _ = pc.popcorn_kernel_matrix(Pd, kern, precision, schedule="tune")
    Ka, _ = pc.popcorn_kernel_matrix(Pd, kern, precision, schedule="auto")
    torch.cuda.synchronize()
    if precision == "fp32":
        assert torch.equal(Ks, Kf) and torch.equal(ds, df)
        Ko = oracle.kernel_matrix(P, kern)
        tol = 1e-6 if kern["kind"] == "gaussian" else 2e-6 * np.abs(Ko) + 1e-6 * np.abs(Ko).max()
        assert np.all(np.abs(Kf.cpu().numpy() - Ko) <= tol)
    else:
        scale = float(Ks.abs().max())
        assert float((Ks - Kf).abs().max()) <= 1e-5 * scale
    assert torch.equal(Kt, Ks) or torch.equal(Kt, Kf)
    assert torch.equal(Ka, Kt)                       # auto takes the cached tuned choice


@pytest.mark.parametrize("n", [700, 1500])
def test_kernel_matrix_gaussian_norm_expansion(pc, n):
    """Images-shaped points with the Gaussian sigma = 28: the largest row norm is about 67, so
    the norm expansion's error bound 4 sqrt(d) u max_i r_i / sigma^2 (~6e-7) is below 1e-6 and
    the FP32 build forms distances by Eq. 12.  K still matches the oracle's coordinate-
    difference K within 1e-6 absolute (the FP32 Gaussian bar), is symmetric, and has diag 1;
    a fit's objective matches the oracle's to 1e-6."""
    wl = synth.workload("images", scale=n / 70000)
    P = _dev(wl.P)
    K, kd = pc.popcorn_kernel_matrix(P, wl.kernel)
    torch.cuda.synchronize()
    Kg = K.cpu().numpy().astype(np.float64)
    Ko = oracle.kernel_matrix(wl.P, wl.kernel)
    assert np.max(np.abs(Kg - Ko)) <= 1e-6
    assert np.array_equal(Kg, Kg.T) and np.all(np.diag(Kg) == 1.0)
    r = pc.popcorn_fit(P, wl.k, wl.kernel, _dev(wl.init_labels), max_iter=5, check_convergence=False)
    assert rel_err(r["objective"], oracle.objective(Ko, r["labels"].cpu().numpy(), wl.k)) <= FP32_OBJ_REL
