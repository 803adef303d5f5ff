"""CSSVDP-LSQR (Algorithm 2) on rank-deficient, infinitely ill-conditioned sparse problems with the
shapes, ranks and densities of the paper's Table C.1 (synthetic stand-ins: exact integer column
dependences, nonzero singular values spread over ~6 decades; b = A x_true, a consistent system).

What the paper's Section 4.4 and Theorems 3.1 / 3.4 fix, checked here:
  * the truncated SVD of the sketch recovers rank(A) (LAPACK's rank of the dense matrix);
  * cond(A P) stays small (the paper observes 3 to 6) although cond(A) is infinite;
  * LSQR on A P converges to the minimum-norm least-squares solution A^+ b (LAPACK lstsq);
  * the oracle's CSSVDP-LSQR, on the smaller shapes, recovers the same rank and solution.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import table_c1_problem

pytestmark = pytest.mark.gpu

SMALL = ["GL7d11", "rel6", "ch8-8-b1", "shar_te2-b1"]
LARGER = ["aa4T", "rel7", "ch8-8-b2"]


@pytest.fixture(scope="module")
def csls():
    from paper_2409_15818_gb300 import build
    build.build()
    from paper_2409_15818_gb300 import csls as mod
    return mod


def _solve(csls, p, seed, prec="f64"):
    A = csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)
    F = csls.csls_factor(A, seed=seed, variant="svd", prec=prec)
    x, rep = csls.csls_solve(F, A, torch.tensor(p.b[0], device="cuda"), variant="svd", tol=1e-14, maxit=500)
    return F, x.cpu().numpy(), rep


@pytest.mark.parametrize("name,prec", [(nm, "f64") for nm in SMALL + LARGER] +
                         [("rel6", "f64emu"), ("ch8-8-b2", "f64emu")])
def test_cssvdp_recovers_rank_and_min_norm_solution(csls, name, prec):
    p = table_c1_problem(name)
    Ad = p.dense()
    rank = np.linalg.matrix_rank(Ad)
    assert rank == p.info["rank"]
    F, x, rep = _solve(csls, p, seed=3, prec=prec)
    assert rep["status"] == 0 and rep["istop"] in (1, 2)
    assert rep["r"] == rank
    assert rep["cond_est"] < 10
    b = p.b[0]
    x_mn = np.linalg.lstsq(Ad, b, rcond=None)[0]
    assert np.linalg.norm(Ad @ x - b) <= 1e-11 * np.linalg.norm(b)
    # x lies in the row space (P = V_r Sigma_r^-1): it is the minimum-norm solution, determined to
    # ~cond_r(A) u with cond_r = sigma_1 / sigma_r ~ 1e5..1e6 here and u the factorisation's unit
    # roundoff (2^-53, or 2^-38 for the emulated products: their error tilts span(V_r) by ~u cond_r)
    sv = np.linalg.svd(Ad, compute_uv=False)
    kappa_r = sv[0] / sv[rank - 1]
    u = 2.0 ** -53 if prec == "f64" else 2.0 ** -38
    assert np.linalg.norm(x - x_mn) <= max(1e-10, 50 * kappa_r * u) * np.linalg.norm(x_mn)


@pytest.mark.parametrize("name", SMALL)
def test_cssvdp_rank_deficient_matches_oracle(csls, name):
    p = table_c1_problem(name)
    s = min(4 * p.n, p.m)
    F, x, rep = _solve(csls, p, seed=5)
    fac, xo, _ = oracle.csqrp_lsqr(p, p.b[0], s=s, seed=5, variant="svd", tol=1e-14, maxit=500)
    assert fac["r"] == rep["r"]
    # P = V_r Sigma_r^-1 with orthonormal V_r: its column norms are 1 / sigma_k
    sig = 1.0 / np.linalg.norm(F.P().cpu().numpy(), axis=0)
    np.testing.assert_allclose(np.sort(sig)[::-1], fac["sigma"][: fac["r"]], rtol=1e-8)
    Ad = p.dense()
    assert np.linalg.norm(Ad @ (x - xo)) <= 1e-10 * np.linalg.norm(Ad @ xo)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
