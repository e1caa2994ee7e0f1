"""Seeded synthetic inputs for Kernel K-means.

This module only draws random numbers: point clouds shaped like the workloads
the method is evaluated on, and the random initial labels of Alg. 2 (line 3:
"assign each point a random cluster").  It holds none of the method's
arithmetic (no kernel function, no distance, no reduction), so both the FP64
oracle and the CUDA path may consume what it produces without sharing any
computation.

All generators use numpy's PCG64 (``numpy.random.default_rng``), whose output
is fixed by the published algorithm and therefore identical on x86_64 and
aarch64 hosts.  Points are returned as C-contiguous float32 arrays, padded with
zero columns to ``d_pad`` where a workload asks for padding; the FP64 oracle
reads exactly these float32 values (widened), so both sides see the same data.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "gaussian_blobs",
    "rings",
    "sparse_images",
    "mixture_varied_sigma",
    "init_labels",
    "small_integer_points",
    "batched_instances",
    "workload",
    "WORKLOADS",
]


@dataclasses.dataclass
class Workload:
    """One clustering problem: points, k, kernel, initial labels and loop mode."""

    name: str
    P: np.ndarray            # (n, d) float32, row-major
    k: int
    kernel: dict             # {"kind": "linear"|"polynomial"|"gaussian", gamma, coef0, degree, sigma}
    init_labels: np.ndarray  # (n,) int32 in [0, k)
    max_iter: int
    check_convergence: bool
    precision: str = "fp32"  # K-build precision: fp32 | bf16 | bf16x3 | fp8
    store_k: bool = True
    tol: float = 0.0

    @property
    def n(self) -> int:
        return int(self.P.shape[0])

    @property
    def d(self) -> int:
        return int(self.P.shape[1])


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def init_labels(n: int, k: int, seed: int) -> np.ndarray:
    """Uniform random labels in [0, k) (0-based form of "a random integer between 1 and k")."""
    return _rng(seed).integers(0, k, size=n, dtype=np.int64).astype(np.int32)


def gaussian_blobs(n: int, d: int, centers: int, seed: int, *, box: float = 10.0,
                   sigma: float = 1.0) -> np.ndarray:
    """Isotropic Gaussian blobs, centres uniform in [-box, box]^d, equal weights."""
    g = _rng(seed)
    C = g.uniform(-box, box, size=(centers, d))
    which = np.arange(n) % centers
    g.shuffle(which)
    X = C[which] + sigma * g.standard_normal(size=(n, d))
    return np.ascontiguousarray(X, dtype=np.float32)


def rings(n: int, radii=(1.0, 2.0, 3.0, 4.0), noise: float = 0.1, seed: int = 0,
          d_pad: int = 8) -> np.ndarray:
    """Concentric rings in the plane (equal counts), radial Gaussian noise, zero-padded to d_pad."""
    g = _rng(seed)
    r_idx = np.arange(n) % len(radii)
    g.shuffle(r_idx)
    theta = g.uniform(0.0, 2.0 * math.pi, size=n)
    r = np.asarray(radii, dtype=np.float64)[r_idx] + noise * g.standard_normal(size=n)
    X = np.zeros((n, d_pad), dtype=np.float64)
    X[:, 0] = r * np.cos(theta)
    X[:, 1] = r * np.sin(theta)
    return np.ascontiguousarray(X, dtype=np.float32)


def sparse_images(n: int, d: int = 784, zero_frac: float = 0.8, seed: int = 0) -> np.ndarray:
    """Image-shaped rows: integers 0..255 divided by 255, with zero_frac of each row zeroed at random."""
    g = _rng(seed)
    X = g.integers(0, 256, size=(n, d), dtype=np.int64).astype(np.float64) / 255.0
    nz = int(round(zero_frac * d))
    # zero a random subset of exactly nz entries in every row
    keys = g.random(size=(n, d))
    cols = np.argpartition(keys, nz - 1, axis=1)[:, :nz] if nz > 0 else np.zeros((n, 0), np.int64)
    np.put_along_axis(X, cols, 0.0, axis=1)
    return np.ascontiguousarray(X, dtype=np.float32)


def mixture_varied_sigma(n: int, d: int, centers: int, seed: int, *, center_std: float = 2.0,
                         sigma_lo: float = 0.5, sigma_hi: float = 1.5) -> np.ndarray:
    """Gaussian mixture: centres ~ N(0, center_std^2 I), per-component sigma ~ U[lo, hi], equal weights."""
    g = _rng(seed)
    C = center_std * g.standard_normal(size=(centers, d))
    s = g.uniform(sigma_lo, sigma_hi, size=centers)
    which = np.arange(n) % centers
    g.shuffle(which)
    X = C[which] + s[which, None] * g.standard_normal(size=(n, d))
    return np.ascontiguousarray(X, dtype=np.float32)


def small_integer_points(n: int, d: int, seed: int, lo: int = -2, hi: int = 2) -> np.ndarray:
    """Points with small integer coordinates: every linear and polynomial kernel entry is exact in FP32."""
    g = _rng(seed)
    return np.ascontiguousarray(g.integers(lo, hi + 1, size=(n, d)), dtype=np.float32)


def _poly(gamma=1.0, coef0=1.0, degree=2):
    return {"kind": "polynomial", "gamma": float(gamma), "coef0": float(coef0), "degree": int(degree),
            "sigma": 1.0}


def _gauss(sigma, gamma=1.0):
    return {"kind": "gaussian", "gamma": float(gamma), "coef0": 0.0, "degree": 1, "sigma": float(sigma)}


def batched_instances(count: int = 256, seed: int = 0, n_lo: int = 500, n_hi: int = 8000,
                      precision: str = "fp32", max_iter: int = 30) -> list:
    """Many independent instances of uneven size: n ~ U[n_lo, n_hi], d in {8, 32, 64}, k ~ U[4, 64].

    Each instance is a k-centre Gaussian mixture (centres in [-5, 5]^d, sigma 1); kernels
    alternate polynomial(1, 1, 2) and Gaussian(sqrt d).
    """
    g = _rng(seed)
    out = []
    for t in range(count):
        n = int(g.integers(n_lo, n_hi + 1))
        d = int(g.choice([8, 32, 64]))
        k = int(g.integers(4, 65))
        k = min(k, n - 1)
        P = gaussian_blobs(n, d, k, seed=seed * 100003 + 7 * t + 1, box=5.0, sigma=1.0)
        kern = _poly(1, 1, 2) if t % 2 == 0 else _gauss(math.sqrt(d))
        lab = init_labels(n, k, seed=seed * 100003 + 7 * t + 2)
        out.append(Workload(f"batch{t}", P, k, kern, lab, max_iter, False, precision))
    return out


def _c1(scale=1.0, seed=0):
    n = max(16, int(2000 * scale))
    P = gaussian_blobs(n, 16, 8, seed=seed + 11, box=10.0, sigma=1.0)
    return Workload("blobs_n2000_d16_k8_poly", P, 8, _poly(1, 1, 2), init_labels(n, 8, seed + 12),
                    30, False, "fp32")


def _c2(scale=1.0, seed=0):
    n = max(16, int(20000 * scale))
    P = rings(n, seed=seed + 21, d_pad=8)
    return Workload("rings_n20000_d8_k4_gauss", P, 4, _gauss(0.5), init_labels(n, 4, seed + 22),
                    100, True, "fp32")


def _c3(scale=1.0, seed=0, precision="fp32"):
    n = max(16, int(70000 * scale))
    P = sparse_images(n, 784, 0.8, seed=seed + 31)
    return Workload(f"images_n70000_d784_k10_gauss_{precision}", P, 10, _gauss(28.0),
                    init_labels(n, 10, seed + 32), 50, False, precision)


def _c5(scale=1.0, seed=0, precision="fp8"):
    n = max(16, int(200000 * scale))
    P = mixture_varied_sigma(n, 128, 100, seed=seed + 51)
    return Workload(f"mixture_n200000_d128_k100_gauss_{precision}", P, 100, _gauss(8.0),
                    init_labels(n, 100, seed + 52), 20, False, precision, store_k=False)


WORKLOADS = {
    "blobs": _c1,       # n=2000, d=16, k=8, polynomial(1,1,2), 30 fixed iterations
    "rings": _c2,       # n=20000, d=2 padded to 8, k=4, Gaussian sigma=0.5, to convergence (<=100)
    "images": _c3,      # n=70000, d=784, k=10, Gaussian sigma=28, 50 fixed iterations
    "mixture": _c5,     # n=200000, d=128, k=100, Gaussian sigma=8, recompute path, 20 iterations
}


def workload(name: str, scale: float = 1.0, seed: int = 0, **kw) -> Workload:
    """Build a named workload; ``scale`` shrinks n for tests (the structure is kept)."""
    return WORKLOADS[name](scale=scale, seed=seed, **kw)
