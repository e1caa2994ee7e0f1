"""GPU parity of K-means++ seeding (popcorn_kmeanspp) against the FP64 oracle (oracle/seeding.py).

Both sides take the same draws u, so the chosen points are compared one by one.  Both take
the sampling decision in FP64 but add the running sums in different orders, so a draw that
lands within rounding of a boundary between two points may pick the neighbour: at the first
point where the sequences differ, the GPU's choice must still be a valid draw for u_t (the
oracle's running sum brackets u_t W within 1e-9 W), and the comparison stops there (the later
steps depend on it).  Labels are each point's nearest chosen point: equal to the oracle's
for the same centers, except where two chosen points are equally near within rounding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle.seeding import kmeanspp  # noqa: E402


@pytest.fixture(scope="module")
def pc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_05587_gb300 as mod
    return mod


def _gauss(s):
    return {"kind": "gaussian", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": s}


POLY2 = {"kind": "polynomial", "gamma": 1.0, "coef0": 1.0, "degree": 2, "sigma": 1.0}
LINEAR = {"kind": "linear", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 1.0}


def _check_against_oracle(P, K, k, u, got_centers, got_labels):
    ref = kmeanspp(K, k, u)
    n = K.shape[0]
    diag = np.diag(K)
    for t in range(k):
        if got_centers[t] == ref["centers"][t]:
            continue
        # the first difference: the GPU's point must be a valid draw for u_t given the same
        # earlier points (identical so far)
        assert t >= 1
        prev = got_centers[:t]
        D = np.min(np.maximum(diag[:, None] - 2 * K[:, prev] + diag[prev][None, :], 0.0), axis=1)
        W = D.sum()
        run = np.cumsum(D)
        c = got_centers[t]
        lo = run[c - 1] if c > 0 else 0.0
        assert D[c] > 0 and lo - 1e-9 * W <= u[t] * W <= run[c] + 1e-9 * W
        return t
    # same centers: labels are the nearest chosen point, up to rounding ties
    if k == 1:
        assert np.all(got_labels == 0)
        return k
    dist = np.maximum(diag[:, None] - 2 * K[:, got_centers] + diag[got_centers][None, :], 0.0)
    best = np.argmin(dist, axis=1)
    part = np.partition(dist, 1, axis=1)
    tie = (part[:, 1] - part[:, 0]) <= 1e-9 * np.maximum(np.abs(part[:, 0]), np.abs(diag))
    assert np.all((got_labels == best) | tie)
    assert np.array_equal(got_labels[got_centers], np.arange(k))
    return k


CASES = [
    # (name, n, d, k, kernel, seed)
    ("blobs", 2000, 16, 8, POLY2, 1),
    ("tiny", 5, 3, 3, _gauss(1.0), 2),                 # fewer points than SMs
    ("k1", 300, 4, 1, _gauss(1.0), 3),
    ("kn", 40, 2, 40, LINEAR, 4),                      # every point chosen
    ("rings", 5000, 8, 4, _gauss(0.5), 5),
    ("images_tenth", 7000, 784, 10, _gauss(28.0), 6),
    ("k100", 3000, 12, 100, _gauss(2.0), 7),
]


@pytest.mark.parametrize("name,n,d,k,kern,seed", CASES)
def test_seeding_is_the_oracle_draw_for_draw(pc, name, n, d, k, kern, seed):
    if name == "images_tenth":
        P = synth.workload("images", scale=0.1).P
    elif name == "rings":
        P = synth.workload("rings", scale=0.25).P
    else:
        P = synth.gaussian_blobs(n, d, max(k, 2), seed=seed, box=3.0)
    n = P.shape[0]
    u = np.random.default_rng(seed + 50).random(k)
    r = pc.popcorn_kmeanspp(torch.from_numpy(P).cuda(), k, kern, u)
    labels = r["labels"].cpu().numpy()
    assert labels.min() >= 0 and labels.max() < k
    K = oracle.kernel_matrix(P, kern)
    _check_against_oracle(P, K, k, u, r["centers"].astype(np.int64), labels.astype(np.int64))


def test_host_and_device_buffers_and_repeat_calls_agree(pc):
    P = synth.gaussian_blobs(3000, 6, 12, seed=11, box=3.0)
    u = np.random.default_rng(9).random(12)
    a = pc.popcorn_kmeanspp(P, 12, _gauss(1.5), u)                                   # host in and out
    b = pc.popcorn_kmeanspp(torch.from_numpy(P).cuda(), 12, _gauss(1.5), torch.from_numpy(u).cuda())
    c = pc.popcorn_kmeanspp(torch.from_numpy(P).cuda(), 12, _gauss(1.5), u)
    assert isinstance(a["labels"], np.ndarray)
    assert np.array_equal(a["labels"], b["labels"].cpu().numpy())
    assert np.array_equal(b["labels"].cpu().numpy(), c["labels"].cpu().numpy())
    assert np.array_equal(a["centers"], b["centers"]) and np.array_equal(b["centers"], c["centers"])


def test_coincident_points_fall_back_to_uniform_draws(pc):
    P = np.ones((500, 4), dtype=np.float32)
    r = pc.popcorn_kmeanspp(P, 3, _gauss(1.0), np.array([0.1, 0.5, 0.999]))
    assert r["centers"].tolist() == [50, 250, 499]
    assert np.all(r["labels"] == 0)


def test_seeded_fit_runs_and_starts_lower_than_random_labels(pc):
    """K-means++ labels feed popcorn_fit; on well-separated blobs they start from a lower
    objective than uniform random labels."""
    wl = synth.workload("blobs")
    u = np.random.default_rng(3).random(wl.k)
    s = pc.popcorn_kmeanspp(torch.from_numpy(wl.P).cuda(), wl.k, wl.kernel, u)
    K = oracle.kernel_matrix(wl.P, wl.kernel)
    seeded = s["labels"].cpu().numpy()
    assert oracle.objective(K, seeded, wl.k) < oracle.objective(K, wl.init_labels, wl.k)
    r = pc.popcorn_fit(torch.from_numpy(wl.P).cuda(), wl.k, wl.kernel, s["labels"], max_iter=30)
    o = oracle.fit(K, wl.k, seeded, 30)
    assert r["iterations"] == o["iterations"]
    assert abs(r["objective"] - o["objective"]) <= 1e-6 * abs(o["objective"])
