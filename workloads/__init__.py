"""Seeded synthetic inputs for the count-sketch preconditioned LSQR path.

This package only builds problems (a CSR matrix A, right-hand sides b and the
metadata needed to evaluate a random-feature solution). It contains none of the
solver's arithmetic: no sketch, no factorisation, no Krylov step. Both the CUDA
path's tests and the CPU oracle's tests draw their inputs from here.
"""
from .rng import splitmix_uniform, splitmix_normal
from .rfm import RFMProblem, poisson2d, poisson3d, rfm_row_descriptors, RFM_ROW_DTYPE
from .synthetic import (scaled_random_sparse, batched_instances, config_problem, rank_deficient_sparse,
                        table_c1_problem, TABLE_C1_SHAPES)

__all__ = [
    "splitmix_uniform", "splitmix_normal", "RFMProblem", "poisson2d", "poisson3d",
    "scaled_random_sparse", "batched_instances", "config_problem", "rank_deficient_sparse", "table_c1_problem",
    "TABLE_C1_SHAPES", "rfm_row_descriptors", "RFM_ROW_DTYPE",
]
