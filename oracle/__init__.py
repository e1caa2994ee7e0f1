"""FP64 CPU oracle for Kernel K-means -- test infrastructure, not a product path.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs may import this package.  See ``oracle/kkmeans.py`` (the method) and
``oracle/seeding.py`` (K-means++ seeding) for what they compute and which passages of
the paper each function follows.
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
from .seeding import kmeanspp  # noqa: F401,E402
