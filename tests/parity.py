"""Shared parity rules for GPU-vs-oracle tests (no GPU needed to import).

Labels: equal except at points whose oracle margin (second-best minus best
distance) is below ``rel * scale_i``, scale_i = max(|best D_i|, K_ii).
Objective: relative error at most ``obj_rel``.
"""
import numpy as np

FP32_LABEL_REL = 1e-6      # margin exemption for the FP32 path
FP32_OBJ_REL = 1e-6        # objective relative error for the FP32 path


def label_mismatches(gpu_labels, oracle_step, rel=FP32_LABEL_REL):
    """Returns (non-exempt mismatches, exempt mismatches) of the new labels of one step."""
    gpu_labels = np.asarray(gpu_labels)
    mism = gpu_labels != oracle_step["labels"]
    exempt = oracle_step["margin"] < rel * oracle_step["scale"]
    return int((mism & ~exempt).sum()), int((mism & exempt).sum())


def rel_err(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _oracle_rows(args):
    import oracle

    P, kern, r0, r1 = args
    return oracle.kernel_matrix(P[r0:r1], kern, Q=P)


def oracle_kernel_matrix(P, kern, workers=None):
    """oracle.kernel_matrix(P, kern), its row blocks computed by a pool of spawned processes.

    Every row of the oracle's K depends only on that row's point and all of P, so the
    blocks are exactly the rows the one-process call returns; the pool only spreads them
    over the host's cores (spawn, never fork: the parent may already hold a CUDA context).
    """
    import concurrent.futures as cf
    import multiprocessing as mp
    import os

    P = np.ascontiguousarray(P)
    n = P.shape[0]
    workers = workers or min(16, os.cpu_count() or 1)
    if n < 4000 or workers == 1:
        import oracle
        return oracle.kernel_matrix(P, kern)
    bounds = np.linspace(0, n, 4 * workers + 1).astype(int)
    out = np.empty((n, n), dtype=np.float64)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        jobs = [(P, kern, int(bounds[i]), int(bounds[i + 1])) for i in range(len(bounds) - 1)]
        for (_, _, r0, r1), block in zip(jobs, ex.map(_oracle_rows, jobs)):
            out[r0:r1] = block
    return out
