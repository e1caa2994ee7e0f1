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
