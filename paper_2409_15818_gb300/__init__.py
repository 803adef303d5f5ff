"""GB300-native count-sketch preconditioned LSQR (CSQRP-LSQR / CSSVDP-LSQR).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/csls.h``); ``csls`` is its thin Python binding.
"""
from . import csls
from .csls import (Csr, Factor, CslsError, CslsSolve, make_opts, solve, csls_factor, csls_solve, csls_sketch,
                   csls_precond_apply, csls_spmv, csls_solve_backward, csls_status_string)

__all__ = ["csls", "Csr", "Factor", "CslsError", "CslsSolve", "make_opts", "solve", "csls_factor", "csls_solve",
           "csls_sketch", "csls_precond_apply", "csls_spmv", "csls_solve_backward", "csls_status_string"]
