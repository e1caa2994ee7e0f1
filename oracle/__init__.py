"""FP64 CPU oracle for Kernel K-means -- test infrastructure, not a product path.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  See ``oracle/kkmeans.py`` for what it computes
and which passages of the paper each function follows.
"""
from .kkmeans import (  # noqa: F401
    KIND_GAUSSIAN,
    KIND_LINEAR,
    KIND_POLYNOMIAL,
    distances,
    fit,
    kernel_matrix,
    objective,
    selection_matrix,
    step,
)
