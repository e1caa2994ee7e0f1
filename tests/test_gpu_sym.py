"""GPU parity of the symmetric pass (popcorn_fit with a stored FP32 K, k_pass = 1).

The pass reads only the 128 x 128 blocks on and above the diagonal: a block's row
sums give one part of S_ic for its rows and, by K's symmetry, its column sums the
part of its columns' rows; a fold kernel adds the parts.  So one pass from given
labels must be the oracle's step exactly as the full-square pass is (labels equal
except near-ties, objective within the FP32 bar), and whole fits must agree with the
full-square pass up to FP32 summation order.  The cases cover a single ragged block,
ragged n over several blocks, n a multiple of 128, k up to its bound (32), a kernel
that is not positive semi-definite (symmetry is all the pass needs) and many blocks,
each with every super-tile edge (1, 2, 3, 4, 8: a super-tile's row and column sums are
kept over its a x a blocks before they are stored; an edge the register file does not
allow falls back to the full square).  k <= 8 with an edge of 1 runs the branch form
(register sums per cluster); otherwise the sorted form runs (every block's labels
sorted each pass, columns and rows walked cluster by cluster, the sums in registers
over the super-tile).  The images workload runs through it
at a tenth of its size against the full oracle step (FP32 build and the packed
tensor-core BF16X3 build), and at full size (n = 70,000, 547 blocks per side) on
sampled rows of E = K V^T that the oracle computes row by row, with every row's
argmin re-derived from E.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.parity import FP32_OBJ_REL, label_mismatches, oracle_kernel_matrix, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


def _gauss(s):
    return {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": s}


POLY2 = {"kind": "polynomial", "gamma": 1.0, "coef0": 1.0, "degree": 2, "sigma": 1.0}
POLY3_NEG = {"kind": "polynomial", "gamma": 0.5, "coef0": -1.0, "degree": 3, "sigma": 1.0}   # not PSD

CASES = [
    # (n, d, k, kernel, seed)
    (97, 3, 3, _gauss(1.0), 1),          # one block, ragged
    (333, 5, 4, POLY2, 2),               # three blocks, ragged
    (1030, 9, 8, _gauss(2.0), 3),        # ragged (n % 4 = 2)
    (2001, 6, 2, _gauss(1.5), 4),
    (1280, 4, 8, _gauss(1.0), 6),        # n a multiple of 128, k at the bound
    (700, 3, 5, POLY3_NEG, 7),           # negative entries: symmetry suffices
    (9001, 4, 5, _gauss(1.0), 5),        # 71 blocks per side
    (1100, 7, 12, _gauss(2.0), 8),       # k > 8: the sorted form at every edge; ragged
    (2500, 5, 16, _gauss(1.5), 9),
    (3000, 6, 10, POLY2, 10),
    (9001, 4, 16, _gauss(1.0), 11),
    (2000, 5, 24, _gauss(1.5), 12),
    (4099, 6, 32, _gauss(2.0), 13),      # k at the bound (32), n % 128 = 3
]


def _sorted_max_a(k):
    """Widest super-tile of the sorted form: its consumer warps (two a block row, two a
    block column; above an edge of 4 each warp owns two block rows or columns), holding
    2 KMAX register sums a lane per block row, must fit the register file (KMAX = 12, 16,
    32 for k up to 12, 16, 32)."""
    return 8 if k <= 12 else 4 if k <= 16 else 3


@pytest.mark.parametrize("sym_tile", [0, 1, 2, 3, 4, 8])
@pytest.mark.parametrize("n,d,k,kern,seed", CASES)
def test_symmetric_pass_is_the_oracle_step(pc, n, d, k, kern, seed, sym_tile):
    P = synth.gaussian_blobs(n, d, k, seed=seed, box=3.0)
    lab = synth.init_labels(n, k, seed=seed + 100)
    r = pc.popcorn_fit(torch.from_numpy(P).cuda(), k, kern, torch.from_numpy(lab).cuda(), max_iter=1,
                       check_convergence=False, k_pass="symmetric", sym_tile=sym_tile)
    # a forced super-tile wider than the register file allows falls back to the full square
    if sym_tile <= _sorted_max_a(k):
        assert r["info"]["k_pass_used"] == 1
    else:
        assert r["info"]["k_pass_used"] == 2
    if sym_tile and r["info"]["k_pass_used"] == 1:
        assert r["info"]["schedule"][0] == sym_tile
    Ko = oracle.kernel_matrix(P, kern)
    st = oracle.step(Ko, lab, k)
    got = r["labels"].cpu().numpy()
    bad, _ = label_mismatches(got, st)
    assert bad == 0
    assert rel_err(r["objective"], oracle.objective(Ko, got, k)) <= FP32_OBJ_REL


@pytest.mark.parametrize("n,d,k,kern,seed", CASES)
def test_symmetric_fit_matches_full_square(pc, n, d, k, kern, seed):
    P = torch.from_numpy(synth.gaussian_blobs(n, d, k, seed=seed, box=3.0)).cuda()
    lab = torch.from_numpy(synth.init_labels(n, k, seed=seed + 200)).cuda()
    a = pc.popcorn_fit(P, k, kern, lab, max_iter=12, check_convergence=False, history=True, k_pass="symmetric")
    b = pc.popcorn_fit(P, k, kern, lab, max_iter=12, check_convergence=False, history=True, k_pass="full")
    Ja, Jb = np.array(a["info"]["J_history"]), np.array(b["info"]["J_history"])
    same = np.mean(a["labels"].cpu().numpy() == b["labels"].cpu().numpy())
    if same == 1.0:
        assert np.all(np.abs(Ja - Jb) <= FP32_OBJ_REL * np.abs(Jb))
        assert rel_err(a["objective"], b["objective"]) <= FP32_OBJ_REL
    else:
        # a near-tie flipped one way under one summation order: the trajectories may part,
        # but each objective must still be that of its labels
        assert same >= 0.99
        Ko = oracle.kernel_matrix(P.cpu().numpy(), kern)
        for r in (a, b):
            assert rel_err(r["objective"], oracle.objective(Ko, r["labels"].cpu().numpy(), k)) <= FP32_OBJ_REL


def test_symmetric_rings_bench_size_matches_full_square(pc):
    """The bench workload (rings, n = 20,000: 157 blocks per side, k = 4) to
    convergence: the symmetric and the full-square pass reach the same labels in the
    same number of passes, objectives within the FP32 bar."""
    wl = synth.workload("rings")
    P = torch.from_numpy(wl.P).cuda()
    L0 = torch.from_numpy(wl.init_labels).cuda()
    a = pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=wl.max_iter, k_pass="symmetric")
    b = pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=wl.max_iter, k_pass="full")
    assert a["info"]["converged"] == 1 and b["info"]["converged"] == 1
    assert a["iterations"] == b["iterations"]
    assert np.array_equal(a["labels"].cpu().numpy(), b["labels"].cpu().numpy())
    assert rel_err(a["objective"], b["objective"]) <= FP32_OBJ_REL


@pytest.mark.parametrize("name,sym_tile", [("rings", 0), ("rings", 2), ("images", 4)])
def test_symmetric_pass_is_deterministic(pc, name, sym_tile):
    """No atomics: every partial is written once and folded in slot order, so runs
    agree bit for bit."""
    wl = synth.workload(name, scale=0.3 if name == "rings" else 0.05)
    P = torch.from_numpy(wl.P).cuda()
    L0 = torch.from_numpy(wl.init_labels).cuda()
    runs = [pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=10, check_convergence=False, history=True,
                           k_pass="symmetric", sym_tile=sym_tile) for _ in range(3)]
    for r in runs[1:]:
        assert r["info"]["J_history"] == runs[0]["info"]["J_history"]
        assert r["objective"] == runs[0]["objective"]
        assert np.array_equal(r["labels"].cpu().numpy(), runs[0]["labels"].cpu().numpy())


def test_symmetric_pass_launches_and_fallback(pc):
    """k_pass = "symmetric" runs the label sort, the stream and the fold (two launches more
    per pass than the full square; the branch form, k <= 8 with a super-tile edge of 1,
    one more).  "auto" reads the full square below 8,192 points (K fits L2 and a pass is
    launch-bound, so at this size the whole fit runs in one launch) and takes the symmetric
    pass from there on.  Above the cluster bound (32) both fall back to the full-square pass,
    with results identical to it; a half-precision K takes the sorted form on the half
    layout."""
    P = torch.from_numpy(synth.gaussian_blobs(600, 3, 6, seed=9, box=3.0)).cuda()
    lab = torch.from_numpy(synth.init_labels(600, 6, seed=19)).cuda()
    a = pc.popcorn_fit(P, 6, _gauss(1.0), lab, max_iter=5, check_convergence=False, k_pass="symmetric")
    br = pc.popcorn_fit(P, 6, _gauss(1.0), lab, max_iter=5, check_convergence=False, k_pass="symmetric",
                        sym_tile=1)
    b = pc.popcorn_fit(P, 6, _gauss(1.0), lab, max_iter=5, check_convergence=False, k_pass="full")
    auto = pc.popcorn_fit(P, 6, _gauss(1.0), lab, max_iter=5, check_convergence=False)
    assert a["info"]["k_pass_used"] == 1 and br["info"]["k_pass_used"] == 1
    assert b["info"]["k_pass_used"] == 2 and auto["info"]["k_pass_used"] == 3   # one-launch fit
    assert rel_err(auto["objective"], b["objective"]) <= FP32_OBJ_REL
    assert a["info"]["kernel_launches"] == b["info"]["kernel_launches"] + 2 * (a["iterations"] + 1)
    assert br["info"]["kernel_launches"] == b["info"]["kernel_launches"] + br["iterations"] + 1
    Pb = torch.from_numpy(synth.gaussian_blobs(9000, 3, 6, seed=9, box=3.0)).cuda()
    labb = torch.from_numpy(synth.init_labels(9000, 6, seed=19)).cuda()
    big = pc.popcorn_fit(Pb, 6, _gauss(1.0), labb, max_iter=2, check_convergence=False)
    assert big["info"]["k_pass_used"] == 1
    h = pc.popcorn_fit(P, 6, _gauss(1.0), lab, max_iter=5, check_convergence=False, k_storage="fp16",
                       k_pass="symmetric")
    assert h["info"]["k_pass_used"] == 1
    lab40 = torch.from_numpy(synth.init_labels(600, 40, seed=29)).cuda()
    c = pc.popcorn_fit(P, 40, _gauss(1.0), lab40, max_iter=5, check_convergence=False, k_pass="symmetric")
    d = pc.popcorn_fit(P, 40, _gauss(1.0), lab40, max_iter=5, check_convergence=False, k_pass="full")
    assert c["info"]["kernel_launches"] == d["info"]["kernel_launches"]
    assert c["info"]["k_pass_used"] == 2
    assert np.array_equal(c["labels"].cpu().numpy(), d["labels"].cpu().numpy())
    assert c["objective"] == d["objective"]


def test_full_size_rings_symmetric_pass_is_the_oracle_step(pc):
    """The rings workload at full size (n = 20,000, k = 4: 157 blocks per side, K stored
    block-packed) through the symmetric pass that popcorn_fit picks for it: the first pass
    from the random initial labels, a pass from the structured labels reached after 20
    passes, and the converged labels, each against the oracle's step on the FP64 K
    (labels element by element up to exempt near-ties, J within the FP32 bar)."""
    wl = synth.workload("rings")
    Ko = oracle_kernel_matrix(wl.P, wl.kernel)
    P = torch.from_numpy(wl.P).cuda()
    L0 = torch.from_numpy(wl.init_labels).cuda()

    def fit(t, **kw):
        return pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=t, check_convergence=False, history=True, **kw)

    r1 = fit(1)
    assert r1["info"]["k_pass_used"] == 1
    st = oracle.step(Ko, wl.init_labels, wl.k)
    got = r1["labels"].cpu().numpy()
    assert label_mismatches(got, st)[0] == 0
    assert rel_err(r1["info"]["J_history"][0], st["J"]) <= FP32_OBJ_REL
    assert rel_err(r1["objective"], oracle.objective(Ko, got, wl.k)) <= FP32_OBJ_REL
    a, b = fit(20), fit(21)
    la = a["labels"].cpu().numpy()
    st = oracle.step(Ko, la, wl.k)
    assert label_mismatches(b["labels"].cpu().numpy(), st)[0] == 0
    assert rel_err(b["info"]["J_history"][20], st["J"]) <= FP32_OBJ_REL
    assert b["info"]["changed_history"][20] == int((b["labels"].cpu().numpy() != la).sum())
    c = pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=wl.max_iter, history=True)
    assert c["info"]["converged"] == 1 and c["info"]["k_pass_used"] == 1
    lc = c["labels"].cpu().numpy()
    st = oracle.step(Ko, lc, wl.k)
    assert label_mismatches(lc, st)[0] == 0               # a fixed point of the oracle's step
    assert rel_err(c["objective"], st["J"]) <= FP32_OBJ_REL


@pytest.mark.parametrize("precision,rel", [("fp32", FP32_OBJ_REL), ("bf16x3", 1e-5)])
def test_images_tenth_symmetric_pass_is_the_oracle_step(pc, precision, rel):
    """The images workload at a tenth of its size (n = 7,000, d = 784, k = 10: 55 blocks
    per side) through the symmetric pass with K block-packed by the FP32 build or by the
    tensor-core BF16X3 build: the first pass and a pass from the labels reached after 5
    passes against the oracle's step on the FP64 K (BF16X3 K carries ~1e-6 relative
    error, so its bars are 1e-5)."""
    wl = synth.workload("images", scale=0.1)
    Ko = oracle_kernel_matrix(wl.P, wl.kernel)
    P = torch.from_numpy(wl.P).cuda()
    L0 = torch.from_numpy(wl.init_labels).cuda()

    def fit(t):
        return pc.popcorn_fit(P, wl.k, wl.kernel, L0, max_iter=t, check_convergence=False, history=True,
                              precision=precision, k_pass="symmetric")

    r1 = fit(1)
    assert r1["info"]["k_pass_used"] == 1
    st = oracle.step(Ko, wl.init_labels, wl.k)
    assert label_mismatches(r1["labels"].cpu().numpy(), st, rel=rel)[0] == 0
    assert rel_err(r1["info"]["J_history"][0], st["J"]) <= rel
    a, b = fit(5), fit(6)
    st = oracle.step(Ko, a["labels"].cpu().numpy(), wl.k)
    assert label_mismatches(b["labels"].cpu().numpy(), st, rel=rel)[0] == 0
    assert rel_err(b["info"]["J_history"][5], st["J"]) <= rel
    assert rel_err(b["objective"], oracle.objective(Ko, b["labels"].cpu().numpy(), wl.k)) <= rel


@pytest.mark.parametrize("k_pass", ["auto", "full"])
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_full_size_images_pass_sampled(pc, precision, k_pass):
    """The images workload at full size (n = 70,000, d = 784, k = 10), one pass from the
    initial labels, through the pass the bench times ("auto": the symmetric pass's sorted
    form, K block-packed, 547 blocks per side, super-tiles of 4 x 4) and through the full
    square (K 19.6 GB).  Sampled rows of E = K V^T (first, last, block edges,
    the ragged tail, random rows) against the oracle's K rows; J against the identity
    J = trace K - sum_c sum_{i in L_c} E_ic; and every row's new label against the argmin
    of D = K_ii - 2 E + ||c||^2 rebuilt from E in FP64 (near-ties exempt)."""
    wl = synth.workload("images")
    n, k = wl.n, wl.k
    P = torch.from_numpy(wl.P).cuda()
    L0 = torch.from_numpy(wl.init_labels).cuda()
    E = torch.empty((n, k), dtype=torch.float32, device="cuda")
    r = pc.popcorn_fit(P, k, wl.kernel, L0, max_iter=1, check_convergence=False, history=True,
                       precision=precision, E_out=E, k_pass=k_pass)
    if k_pass == "auto":
        assert r["info"]["k_pass_used"] == 1 and r["info"]["schedule"][0] == 4
    else:
        assert r["info"]["k_pass_used"] == 2
    Eg = E.cpu().numpy().astype(np.float64)
    lab = wl.init_labels.astype(np.int64)
    m = np.bincount(lab, minlength=k).astype(np.float64)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([[0, 1, 127, 128, 129, n - 129, n - 2, n - 1],
                                     rng.choice(n, 40, replace=False)]))
    Kr = oracle.kernel_matrix(wl.P[rows], wl.kernel, Q=wl.P)
    Eo = np.stack([Kr[:, lab == c].sum(axis=1) / m[c] for c in range(k)], axis=1)
    assert np.max(np.abs(Eg[rows] - Eo)) <= 1e-5 * np.abs(Eo).max()
    z = np.array([Eg[lab == c, c].sum() / m[c] for c in range(k)])
    trace = float(n)                                   # Gaussian: K_ii = 1
    J_E = trace - sum(Eg[lab == c, c].sum() for c in range(k))
    assert rel_err(r["info"]["J_history"][0], J_E) <= 1e-6
    D = 1.0 - 2.0 * Eg + z[None, :]
    pred = np.argmin(D, axis=1)
    part = np.partition(D, 1, axis=1)
    exempt = (part[:, 1] - part[:, 0]) < 1e-6 * np.maximum(np.abs(part[:, 0]), 1.0)
    got = r["labels"].cpu().numpy()
    assert int(((got != pred) & ~exempt).sum()) == 0


def test_sorted_form_launches_its_label_sort(pc):
    """The sorted form adds two launches per pass to the full square's one (the per-pass
    sort of every block's labels, then the stream, then the fold)."""
    P = torch.from_numpy(synth.gaussian_blobs(900, 3, 12, seed=4, box=3.0)).cuda()
    lab = torch.from_numpy(synth.init_labels(900, 12, seed=14)).cuda()
    a = pc.popcorn_fit(P, 12, _gauss(1.0), lab, max_iter=4, check_convergence=False, timing=True,
                       k_pass="symmetric")
    b = pc.popcorn_fit(P, 12, _gauss(1.0), lab, max_iter=4, check_convergence=False, timing=True, k_pass="full")
    auto = pc.popcorn_fit(P, 12, _gauss(1.0), lab, max_iter=4, check_convergence=False, timing=True)
    assert auto["info"]["k_pass_used"] == 3          # n < 8,192: the one-launch fit unless forced
    assert a["info"]["k_pass_used"] == 1 and b["info"]["k_pass_used"] == 2
    assert a["info"]["schedule"][3] == 12            # the sorted form's register sums (KMAX)
    assert a["info"]["kernel_launches"] == b["info"]["kernel_launches"] + 2 * (a["iterations"] + 1)
