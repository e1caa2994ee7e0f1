"""The row-sharded form of one assignment pass, on CPU ranks (gloo, world size 2 and 3).

The pass shards by rows of K: rank g owns rows [r_g, r_{g+1}) and builds its row block
of K from all of P (P is replicated).  Per pass, with the labels replicated on every
rank:
  1. local:     E_g = K_g V^T for its rows (the paper's SpMM, Alg. 2 line 7, on a row
                block), and the FP64 partial sums zp_c = sum_{i in L_c, i in g} E_ic;
  2. exchange:  one allreduce (sum) of the k partials -- ||c_c||^2 = zp_c / |L_c|
                (Eq. 14's SpMV, split by rows);
  3. local:     D for its rows (Eq. 11), the row argmin, its part of J and of the change
                count, folded into the same allreduce's successor (a second tiny sum);
  4. exchange:  one allgather of the new labels (n int32) for the next pass's V.
The arithmetic on each shard is the oracle's own (its kernel function, its V), so the
sharded pass must reproduce the oracle's unsharded step: labels (up to near-ties that a
different FP64 summation order may resolve either way), J and the centroid norms to
FP64 rounding.  Every rank of this test is a CPU process; the GPU form of this
exchange is not built on one GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def row_bounds(n, world):
    """Rank g owns rows [b[g], b[g + 1]): contiguous, sizes differing by at most one."""
    return [n * g // world for g in range(world + 1)]


def sharded_step(P, kern, labels, k, rank, world):
    """One pass of the row-sharded Kernel K-means on this rank; returns what every rank holds
    after the pass: the new labels (all n), J(labels), the centroid norms, the change count."""
    n = P.shape[0]
    b = row_bounds(n, world)
    r0, r1 = b[rank], b[rank + 1]
    labels = np.asarray(labels, dtype=np.int64)
    Kg = oracle.kernel_matrix(P[r0:r1], kern, Q=P)               # this rank's row block of K
    V = oracle.selection_matrix(labels, k)                       # replicated (labels are)
    counts = np.bincount(labels, minlength=k)
    Eg = Kg @ V.T                                                # (K V^T) for rows r0..r1
    own = labels[r0:r1]
    zp = np.zeros(k)
    np.add.at(zp, own, Eg[np.arange(r1 - r0), own])              # sum_{i in L_c, i in g} E_ic
    zt = torch.from_numpy(zp)
    dist.all_reduce(zt)                                          # exchange 1: k FP64 sums
    inv = np.where(counts > 0, 1.0 / np.maximum(counts, 1), 0.0)
    cnorm = zt.numpy() * inv                                     # ||c_c||^2 = (1/m_c) sum E_ic
    kdiag = np.array([Kg[i, r0 + i] for i in range(r1 - r0)])
    D = -2.0 * Eg + kdiag[:, None] + cnorm[None, :]
    D[:, counts == 0] = np.inf
    new_own = np.argmin(D, axis=1)
    part = torch.tensor([D[np.arange(r1 - r0), own].sum(), float((new_own != own).sum())], dtype=torch.float64)
    dist.all_reduce(part)                                        # J and the change count
    # exchange 2: the labels, every shard padded to the largest (an all-gather moves equal sizes)
    width = max(b[g + 1] - b[g] for g in range(world))
    mine = torch.full((width,), -1, dtype=torch.int64)
    mine[: r1 - r0] = torch.from_numpy(new_own.astype(np.int64))
    gathered = [torch.empty(width, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, mine)
    new = torch.cat([gathered[g][: b[g + 1] - b[g]] for g in range(world)]).numpy()
    return new, float(part[0]), cnorm, int(part[1])


def _worker(rank, world, port, case, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, d, k, kern, seed, passes = case
        P = synth.gaussian_blobs(n, d, k, seed=seed, box=3.0)
        lab = synth.init_labels(n, k, seed=seed + 1)
        hist = []
        for _ in range(passes):
            new, J, cn, ch = sharded_step(P, kern, lab, k, rank, world)
            hist.append((lab.copy(), new, J, cn, ch))
            lab = new
        out[rank] = hist
        dist.barrier()
    finally:
        dist.destroy_process_group()


CASES = [
    (301, 3, 4, {"kind": "gaussian", "gamma": 1.0, "sigma": 1.5}, 3, 4),
    (257, 5, 6, {"kind": "polynomial", "gamma": 1.0, "coef0": 1.0, "degree": 2}, 5, 3),
]


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=["gauss", "poly2"])
def test_row_sharded_pass_is_the_oracle_step(world, case):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, case, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    n, d, k, kern, seed, passes = case
    P = synth.gaussian_blobs(n, d, k, seed=seed, box=3.0)
    K = oracle.kernel_matrix(P, kern)
    for t in range(passes):
        lab_in = res[0][t][0]
        st = oracle.step(K, lab_in, k)
        for r in range(world):
            src, new, J, cn, ch = res[r][t]
            assert np.array_equal(src, lab_in)                       # every rank held the same labels
            exempt = st["margin"] < 1e-12 * st["scale"]
            assert np.all((new == st["labels"]) | exempt)
            assert J == pytest.approx(st["J"], rel=1e-12)
            nonempty = st["counts"] > 0
            np.testing.assert_allclose(cn[nonempty], st["cnorm"][nonempty], rtol=1e-12, atol=1e-12)
            assert ch == int((new != lab_in).sum())


def test_row_bounds_cover_every_row_once():
    for n in (1, 2, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            b = row_bounds(n, world)
            assert b[0] == 0 and b[-1] == n
            assert all(b[g] <= b[g + 1] for g in range(world))
            assert max(b[g + 1] - b[g] for g in range(world)) - min(b[g + 1] - b[g] for g in range(world)) <= 1
