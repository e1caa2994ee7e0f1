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


def _oracle_rounded(P, kern, storage):
    """The oracle's K, rounded to FP32 (the build's type) and then to the storage type.  The
    GPU's FP32 build differs from the FP32 rounding of the exact K by an FP32 ulp at most, so
    the two half roundings differ only where a half boundary falls inside that ulp (about 1
    entry in 2^13 for FP16): far below the bars below."""
    return _rounded(oracle.kernel_matrix(P, kern).astype(np.float32), storage)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("storage,name,scale", [("fp16", "rings", 0.1), ("bf16", "rings", 0.1),
                                                ("bf16", "blobs", 0.5)])
def test_half_k_first_pass_matches_oracle_on_rounded_k(pc, storage, name, scale):
    wl = synth.workload(name, scale=scale)
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=1, check_convergence=False,
                       k_storage=storage, history=True)
    Kr = _oracle_rounded(wl.P, wl.kernel, storage)
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


# ---------------------------------------------------------------- symmetric pass on a half K
# k_pass="symmetric" stores the packed upper triangle in FP16 / BF16 (the FP32 build's
# triangle, rounded by one pack launch): the same rounded K as the full-square half path,
# half the bytes again, read by the tensor-core form (MMAs of each tile against one-hot
# label operands, FP32 accumulators in TMEM).  Cases span several super-tiles and ragged
# edges (n not a multiple of 128) and both accumulator widths (N = 16 for k <= 16, 32 up
# to 32).

SYM_HALF = [("fp16", "rings", 0.1, None), ("bf16", "rings", 0.1, None), ("bf16", "blobs", 0.5, None),
            ("fp16", "rings", 0.15, 14), ("bf16", "blobs", 0.5, 27)]   # FP16: Gaussian K only (|K| <= 1)


@pytest.mark.parametrize("storage,name,scale,k", SYM_HALF)
def test_half_k_symmetric_first_pass_matches_oracle_on_rounded_k(pc, storage, name, scale, k):
    wl = synth.workload(name, scale=scale)
    k = k or wl.k
    lab = synth.init_labels(wl.P.shape[0], k, seed=8) if k != wl.k else wl.init_labels
    r = pc.popcorn_fit(_dev(wl.P), k, wl.kernel, _dev(lab), max_iter=1, check_convergence=False,
                       k_storage=storage, k_pass="symmetric", history=True)
    assert r["info"]["k_pass_used"] == 1 and r["info"]["sym_form"] == 3
    assert r["info"]["schedule"][3] == (16 if k <= 16 else 32)
    Kr = _oracle_rounded(wl.P, wl.kernel, storage)
    st = oracle.step(Kr, lab, k)
    assert rel_err(r["info"]["J_history"][0], st["J"]) <= 1e-5
    rel = 2.0 ** -11 if storage == "fp16" else 2.0 ** -8
    assert label_mismatches(r["labels"].cpu().numpy(), st, rel=rel)[0] == 0


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_half_k_symmetric_and_full_square_agree(pc, storage):
    """Same rounded K, two reads of it: identical labels at every pass up to summation-order
    near-ties, objectives to 1e-5."""
    wl = synth.workload("rings", scale=0.15)
    kw = dict(max_iter=wl.max_iter, check_convergence=False, k_storage=storage, history=True)
    a = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), k_pass="symmetric", **kw)
    b = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), k_pass="full", **kw)
    assert a["info"]["k_pass_used"] == 1 and b["info"]["k_pass_used"] == 2 and a["info"]["sym_form"] == 3
    Ja, Jb = np.array(a["info"]["J_history"]), np.array(b["info"]["J_history"])
    assert np.all(np.abs(Ja - Jb) <= 1e-5 * np.abs(Jb))


@pytest.mark.parametrize("storage,precision", [("fp16", "bf16"), ("bf16", "bf16"), ("fp16", "bf16x3"),
                                               ("bf16", "bf16x3")])
def test_half_k_from_tensor_core_build_exact_on_small_integers(pc, storage, precision):
    """The tensor-core builds write the half triangle directly.  Points with small integer
    coordinates make every product and every entry of the linear K exact in BF16 and in the
    storage type (|K_ij| <= 36), so one symmetric pass must be the oracle's step on the
    exact K: labels equal, J to FP32 rounding of exact integer sums."""
    rng = np.random.default_rng(21)
    n, k = 3001, 9
    P = rng.integers(-3, 4, size=(n, 4)).astype(np.float32)
    lab = synth.init_labels(n, k, seed=22)
    lin = {"kind": "linear", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 1.0}
    r = pc.popcorn_fit(_dev(P), k, lin, _dev(lab), max_iter=1, check_convergence=False, k_storage=storage,
                       precision=precision, k_pass="symmetric", history=True)
    assert r["info"]["k_pass_used"] == 1 and r["info"]["sym_form"] == 3
    st = oracle.step(oracle.kernel_matrix(P, lin), lab, k)
    assert rel_err(r["info"]["J_history"][0], st["J"]) <= 1e-6
    assert label_mismatches(r["labels"].cpu().numpy(), st, rel=1e-6)[0] == 0


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_half_k_from_bf16x3_build_gaussian(pc, storage):
    """BF16X3 build, half K written by its epilogue (the bench's fast form): one pass against
    the oracle's step on its K rounded to the storage type.  BF16X3 entries carry ~16
    significant bits (relative error ~1e-5 at this sigma), which the J bar allows for."""
    wl = synth.workload("rings", scale=0.15)
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=1, check_convergence=False,
                       k_storage=storage, precision="bf16x3", k_pass="symmetric", history=True)
    assert r["info"]["k_pass_used"] == 1 and r["info"]["sym_form"] == 3
    st = oracle.step(_oracle_rounded(wl.P, wl.kernel, storage), wl.init_labels, wl.k)
    assert rel_err(r["info"]["J_history"][0], st["J"]) <= 5e-5
    rel = 2.0 ** -10 if storage == "fp16" else 2.0 ** -7
    assert label_mismatches(r["labels"].cpu().numpy(), st, rel=rel)[0] == 0


def test_half_k_symmetric_ragged_and_host_buffers(pc):
    P = synth.gaussian_blobs(1001, 5, 3, seed=4, box=3.0)
    lab = synth.init_labels(1001, 7, seed=5)
    kern = {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 2.0}
    a = pc.popcorn_fit(P, 7, kern, lab, max_iter=20, k_storage="bf16", k_pass="symmetric")
    b = pc.popcorn_fit(_dev(P), 7, kern, _dev(lab), max_iter=20, k_storage="bf16", k_pass="symmetric")
    assert np.array_equal(a["labels"], b["labels"].cpu().numpy()) and a["objective"] == b["objective"]
    c = pc.popcorn_fit(_dev(P), 7, kern, _dev(lab), max_iter=20, k_storage="bf16", k_pass="full")
    assert a["info"]["k_pass_used"] == 1 and c["info"]["k_pass_used"] == 2
    assert rel_err(a["objective"], c["objective"]) <= 1e-5


@pytest.mark.parametrize("storage,precision", [("fp16", "fp32"), ("bf16", "fp32"), ("fp16", "bf16x3")])
def test_half_k_symmetric_sampled_rows_at_images_size(pc, storage, precision):
    """Images at full size (n = 70,000, d = 784, k = 10, Gaussian): the automatic choice
    takes the symmetric pass on the half K (the packed triangle, 4.9 GB).  One pass from
    the initial labels: sampled rows of E = K V^T (block edges, the ragged tail, random
    rows) against the oracle's K rows rounded like the stored K; J against the identity
    J = trace K - sum_c sum_{i in L_c} E_ic; every row's new label against the argmin of
    D = K_ii - 2 E + ||c||^2 rebuilt from E in FP64 (near-ties exempt)."""
    wl = synth.workload("images")
    n, k = wl.n, wl.k
    E = torch.empty((n, k), dtype=torch.float32, device="cuda")
    r = pc.popcorn_fit(_dev(wl.P), k, wl.kernel, _dev(wl.init_labels), max_iter=1, check_convergence=False,
                       k_storage=storage, precision=precision, history=True, E_out=E)
    assert r["info"]["k_pass_used"] == 1 and r["info"]["sym_form"] == 3
    Eg = E.cpu().numpy().astype(np.float64)
    lab = wl.init_labels.astype(np.int64)
    m = np.bincount(lab, minlength=k).astype(np.float64)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([[0, 1, 127, 128, 129, n - 129, n - 2, n - 1],
                                     rng.choice(n, 40, replace=False)]))
    # the oracle's rows, through FP32 (the build's type) and then the storage type
    Kr = _rounded(oracle.kernel_matrix(wl.P[rows], wl.kernel, Q=wl.P).astype(np.float32), storage)
    Eo = np.stack([Kr[:, lab == c].sum(axis=1) / m[c] for c in range(k)], axis=1)
    # BF16X3 entries carry ~16 significant bits: a looser bar on the sampled rows
    assert np.max(np.abs(Eg[rows] - Eo)) <= (1e-5 if precision == "fp32" else 5e-5) * np.abs(Eo).max()
    z = np.array([Eg[lab == c, c].sum() / m[c] for c in range(k)])
    trace = float(n)                                   # Gaussian: K_ii = 1, exact in both types
    J_E = trace - sum(Eg[lab == c, c].sum() for c in range(k))
    assert rel_err(r["info"]["J_history"][0], J_E) <= 1e-6
    D = 1.0 - 2.0 * Eg + z[None, :]
    pred = np.argmin(D, axis=1)
    part = np.partition(D, 1, axis=1)
    exempt = (part[:, 1] - part[:, 0]) < 1e-6 * np.maximum(np.abs(part[:, 0]), 1.0)
    got = r["labels"].cpu().numpy()
    assert int(((got != pred) & ~exempt).sum()) == 0


HALF_EDGE_CASES = [
    # (n, d, k, sigma, seed): Gaussian (|K| <= 1, FP16-safe)
    (97, 3, 3, 1.0, 1),          # one block, ragged
    (300, 3, 1, 1.0, 20),        # k = 1
    (1030, 9, 8, 2.0, 3),        # ragged
    (1280, 4, 16, 1.0, 6),       # n a multiple of 128, N = 16 at its bound
    (2000, 5, 24, 1.5, 12),      # N = 32
    (4099, 6, 32, 2.0, 13),      # k at the bound (32), n % 128 = 3
]


@pytest.mark.parametrize("sym_tile", [0, 1, 2, 3, 5, 8])
@pytest.mark.parametrize("n,d,k,sigma,seed", HALF_EDGE_CASES)
def test_half_k_symmetric_every_super_tile_edge(pc, n, d, k, sigma, seed, sym_tile):
    """Every super-tile edge of the tensor-core form: the 2a accumulators of N columns,
    double-buffered, must fit TMEM's 512 columns (a <= 8 for N = 16, a <= 4 for N = 32); a
    larger forced edge falls back to the full square.  Either way one pass is the oracle's
    step on the rounded K."""
    P = synth.gaussian_blobs(n, d, k, seed=seed, box=3.0)
    lab = synth.init_labels(n, k, seed=seed + 100)
    kern = {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": sigma}
    r = pc.popcorn_fit(_dev(P), k, kern, _dev(lab), max_iter=1, check_convergence=False, k_storage="fp16",
                       k_pass="symmetric", sym_tile=sym_tile, history=True)
    amax = 8 if k <= 16 else 4
    if sym_tile <= amax:
        assert r["info"]["k_pass_used"] == 1 and r["info"]["sym_form"] == 3
        if sym_tile:
            assert r["info"]["schedule"][0] == sym_tile
            T = (n + 127) // 128
            assert r["info"]["schedule"][2] == (T + sym_tile - 1) // sym_tile + 1   # slots: Ts + 1
    else:
        assert r["info"]["k_pass_used"] == 2
    st = oracle.step(_oracle_rounded(P, kern, "fp16"), lab, k)
    assert rel_err(r["info"]["J_history"][0], st["J"]) <= 1e-5
    assert label_mismatches(r["labels"].cpu().numpy(), st, rel=2.0 ** -11)[0] == 0


def test_half_k_symmetric_is_deterministic(pc):
    """Fixed block order, fixed MMA order into each accumulator, fixed fold order: repeated
    fits give bit-identical objectives and labels."""
    wl = synth.workload("rings", scale=0.25)
    runs = [pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=10, check_convergence=False,
                           k_storage="bf16", k_pass="symmetric", history=True) for _ in range(3)]
    for r in runs[1:]:
        assert r["info"]["J_history"] == runs[0]["info"]["J_history"]
        assert torch.equal(r["labels"], runs[0]["labels"])


def test_half_k_from_tensor_core_build_auto_choice_and_limits(pc):
    """A half K from a BF16 / BF16X3 build: the automatic read takes the tensor-core symmetric
    form at any n (here n = 2,500, below the FP32 threshold); a read of the full square
    (k > 32, or k_pass = "full") runs on the tensor cores too, as batched mode's one-instance
    stream (k_pass_used 2, schedule[3] = k rounded up to 16), and repeats bit for bit."""
    wl = synth.workload("images", scale=2500 / 70000)
    n = wl.P.shape[0]
    r = pc.popcorn_fit(_dev(wl.P), wl.k, wl.kernel, _dev(wl.init_labels), max_iter=3, check_convergence=False,
                       k_storage="fp16", precision="bf16x3", history=True)
    assert r["info"]["k_pass_used"] == 1 and r["info"]["sym_form"] == 3
    for k, kp in ((40, "auto"), (wl.k, "full")):
        lab = synth.init_labels(n, k, seed=3)
        a = pc.popcorn_fit(_dev(wl.P), k, wl.kernel, _dev(lab), max_iter=2, check_convergence=False,
                           k_storage="bf16", precision="bf16x3", k_pass=kp, history=True)
        assert a["info"]["k_pass_used"] == 2 and a["info"]["schedule"][3] == (k + 15) // 16 * 16
        b = pc.popcorn_fit(_dev(wl.P), k, wl.kernel, _dev(lab), max_iter=2, check_convergence=False,
                           k_storage="bf16", precision="bf16x3", k_pass=kp, history=True)
        assert a["info"]["J_history"] == b["info"]["J_history"]
        assert torch.equal(a["labels"], b["labels"])


@pytest.mark.parametrize("storage,precision,n,k", [("bf16", "fp32", 9001, 40), ("fp16", "bf16x3", 3000, 100),
                                                   ("bf16", "bf16", 2500, 64), ("fp16", "fp32", 8300, 33)])
def test_half_k_full_square_on_tensor_cores(pc, storage, precision, n, k):
    """A half K read as the full square on the tensor cores (k > 32): the FP32 square of the
    build rounded into half tiles, each 128-row block's tiles MMA'd against one-hot label
    operands, one segment, the z reduction and the argmin.  One pass against the oracle's
    step on the oracle's K rounded to the storage type (for the BF16 build, the K of the
    BF16-rounded points)."""
    P = synth.gaussian_blobs(n, 6, 20, seed=k, box=3.0)
    lab = synth.init_labels(n, k, seed=k + 1)
    kern = {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 2.0}
    r = pc.popcorn_fit(_dev(P), k, kern, _dev(lab), max_iter=1, check_convergence=False, k_storage=storage,
                       precision=precision, history=True)
    assert r["info"]["k_pass_used"] == 2 and r["info"]["schedule"][3] == (k + 15) // 16 * 16
    Pu = P
    if precision == "bf16":
        Pu = torch.from_numpy(P).to(torch.bfloat16).to(torch.float64).numpy()
    st = oracle.step(_oracle_rounded(Pu, kern, storage), lab, k)
    bar = 1e-5 if precision == "fp32" else 1e-4
    assert rel_err(r["info"]["J_history"][0], st["J"]) <= bar
    rel = 2.0 ** -10 if storage == "fp16" else 2.0 ** -7
    assert label_mismatches(r["labels"].cpu().numpy(), st, rel=rel)[0] == 0
