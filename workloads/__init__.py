"""Seeded synthetic inputs for the count-sketch preconditioned LSQR path.

This package only builds problems (a CSR matrix A, right-hand sides b and the
metadata needed to evaluate a random-feature solution). It contains none of the
solver's arithmetic: no sketch, no factorisation, no Krylov step. Both the CUDA
path's tests and the CPU oracle's tests draw their inputs from here.
"""
import hashlib

import numpy as np

from .rng import splitmix_uniform, splitmix_normal
from .rfm import RFMProblem, poisson2d, poisson3d, rfm_row_descriptors, RFM_ROW_DTYPE
from .synthetic import (scaled_random_sparse, batched_instances, config_problem, rank_deficient_sparse,
                        table_c1_problem, TABLE_C1_SHAPES)

__all__ = [
    "splitmix_uniform", "splitmix_normal", "RFMProblem", "poisson2d", "poisson3d",
    "scaled_random_sparse", "batched_instances", "config_problem", "rank_deficient_sparse", "table_c1_problem",
    "TABLE_C1_SHAPES", "rfm_row_descriptors", "RFM_ROW_DTYPE", "input_hash",
]


def input_hash(p):
    """SHA-256 of a problem's CSR arrays and right-hand sides (the key of cached oracle results). The
    generators use only IEEE-exact elementwise arithmetic (``detmath``), so the same recipe hashes the same
    on every machine."""
    h = hashlib.sha256()
    for a, dt in ((p.row_ptr, np.int64), (p.col, np.int32), (p.val, np.float64), (p.b, np.float64)):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()
