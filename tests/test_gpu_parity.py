"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs, at sizes the oracle finishes in seconds that still span
several tiles, panels and a ragged tail.

Tolerances:
  * sketch: bit-exact (binary64 and binary32), same hash and ascending-row order;
  * R: relative difference <= 1e-12 on well-conditioned sketches; on the
    ill-conditioned RFM sketches the backward error ||R^T R - SA^T SA|| / ||SA||^2
    is checked instead (the R factor itself is then only determined to about
    cond(SA) * 2^-53);
  * solution: with cond(A) moderate, ||x - x_oracle|| / ||x_oracle|| <= 1e-10;
    on RFM matrices (cond(A) ~ 1e9) x is only determined up to cond(A) * 2^-53,
    so the A-norm ||A (x - x_oracle)|| / ||A x_oracle|| (the norm Theorem 3.3
    bounds) must be <= max(1e-10, 2 x the spread between the two independent
    oracle solvers), and the residual norms must agree to 1e-12 ||b||.
"""
import numpy as np
import pytest
import torch

import oracle
from tests.helpers import CSR, csr_from_dense, random_sparse
from workloads import config_problem, poisson2d, scaled_random_sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csls():
    from paper_2409_15818_gb300 import build
    build.build()
    from paper_2409_15818_gb300 import csls as mod
    return mod


def dev(csls, p):
    return csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)


def gpu_sketch(csls, A, s, seed, prec):
    t = csls.csls_sketch(A, s, seed, prec=prec)
    torch.cuda.synchronize()
    return t.cpu().numpy().T[:s, :]


SKETCH_CASES = {
    "cfg1": lambda: config_problem("cfg1"),
    "ragged_rfm": lambda: poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7),
    "cfg5_slice": lambda: config_problem("cfg5_slice"),
}


@pytest.mark.parametrize("case", list(SKETCH_CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sketch_bit_exact(csls, case, prec):
    p = SKETCH_CASES[case]()
    for s, seed in ((4 * p.n if 4 * p.n < p.m else p.m, 11), (p.m // 3 + 1, 12345)):
        got = gpu_sketch(csls, dev(csls, p), s, seed, prec)
        h, d = oracle.hash_rows(p.m, s, seed)
        want = oracle.sketch(p, s, h, d, np.float64 if prec == "f64" else np.float32)
        assert got.shape == want.shape
        assert np.array_equal(got.view(np.uint64 if prec == "f64" else np.uint32),
                              np.asarray(want).view(np.uint64 if prec == "f64" else np.uint32))


@pytest.mark.parametrize("s", [1, 2, 97])
def test_sketch_degenerate_bucket_counts(csls, s):
    """Very few buckets: every bucket holds many rows (long-segment sort paths)."""
    p = scaled_random_sparse(9000, 30, per_row=3, cond_exp=1.0, seed=3)
    got = gpu_sketch(csls, dev(csls, p), s, 5, "f64")
    h, d = oracle.hash_rows(p.m, s, 5)
    want = oracle.sketch(p, s, h, d)
    assert np.array_equal(got, want)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_factor_r_matches_oracle_well_conditioned(csls):
    rng = np.random.default_rng(21)
    A = random_sparse(3000, 200, 12, rng)   # 200 = 6 panels of 32 + 8, 4 TRSV blocks (ragged)
    F = csls.csls_factor(dev(csls, A), s=800, seed=9)
    R = F.R().cpu().numpy()
    fac = oracle.factor(A, 800, 9)
    assert _rel(R, fac["R"]) < 1e-12
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
    F32 = csls.csls_factor(dev(csls, A), s=800, seed=9, prec="f32")
    R32 = F32.R().cpu().numpy().astype(np.float64)
    R32o = oracle.r_factor(oracle.sketch(A, 800, *oracle.hash_rows(A.m, 800, 9), np.float32))
    assert _rel(R32, R32o) < 1e-5 and _rel(R32, fac["R"]) < 1e-5


def test_factor_backward_error_rfm(csls):
    p = config_problem("cfg1")
    F = csls.csls_factor(dev(csls, p), seed=11)
    R = F.R().cpu().numpy()
    h, d = oracle.hash_rows(p.m, 4 * p.n, 11)
    SA = oracle.sketch(p, 4 * p.n, h, d)
    err = np.linalg.norm(R.T @ R - SA.T @ SA) / np.linalg.norm(SA) ** 2
    assert err < 50 * p.n * 2.0 ** -53
    Ro = oracle.factor(p, 4 * p.n, 11)["R"]
    assert _rel(R, Ro) < 1e-6
    assert F.report["rdiag_min"] > 0 and F.report["s"] == 4 * p.n


def test_precond_apply_and_spmv_pair(csls):
    rng = np.random.default_rng(22)
    A = random_sparse(2500, 150, 9, rng, scale_exp=3.0)
    Ad = dev(csls, A)
    F = csls.csls_factor(Ad, s=600, seed=4)
    R = F.R().cpu().numpy()
    v = rng.standard_normal(150)
    vt = torch.tensor(v, device="cuda")
    z = csls.csls_precond_apply(F, vt).cpu().numpy()
    zt = csls.csls_precond_apply(F, vt, trans=True).cpu().numpy()
    assert _rel(z, oracle.trsv_upper(R, v)) < 1e-12
    assert _rel(zt, oracle.trsv_upper_trans(R, v)) < 1e-12
    x = rng.standard_normal(150)
    u = rng.standard_normal(2500)
    y = csls.csls_spmv(F, Ad, torch.tensor(x, device="cuda")).cpu().numpy()
    g = csls.csls_spmv(F, Ad, torch.tensor(u, device="cuda"), trans=True).cpu().numpy()
    assert _rel(y, oracle.spmv(A, x)) < 1e-14
    assert _rel(g, oracle.spmv_trans(A, u)) < 1e-14


def test_solve_well_conditioned_x_space(csls):
    """cond(A) ~ 1e3: the solution is determined to ~1e-13, so x itself must match."""
    rng = np.random.default_rng(23)
    A = random_sparse(4000, 230, 10, rng, scale_exp=3.0)
    b = rng.standard_normal(4000)
    F = csls.csls_factor(dev(csls, A), s=920, seed=6)
    x, rep = csls.csls_solve(F, dev(csls, A), torch.tensor(b, device="cuda"), tol=1e-14, maxit=400)
    _, xo, info = oracle.csqrp_lsqr(A, b, s=920, seed=6, tol=1e-14, maxit=400)
    assert _rel(x.cpu().numpy(), xo) < 1e-10
    assert rep["istop"] in (1, 2) and abs(rep["iterations"] - info["iterations"]) <= 3
    assert rep["cond_est"] < 10


def _anorm_rel(Ad, x, xo):
    return np.linalg.norm(Ad @ (x - xo)) / np.linalg.norm(Ad @ xo)


@pytest.mark.parametrize("case", ["cfg1", "ragged_rfm"])
def test_solve_rfm_matches_oracle(csls, case):
    p = SKETCH_CASES[case]()
    Ad = p.dense()
    b = p.b[0]
    F = csls.csls_factor(dev(csls, p), seed=11)
    x, rep = csls.csls_solve(F, dev(csls, p), torch.tensor(b, device="cuda"))
    x = x.cpu().numpy()
    fac, xo, info = oracle.csqrp_lsqr(p, b, seed=11)
    x_hh, _ = oracle.hhqr_solve(Ad, b)
    spread = _anorm_rel(Ad, x_hh, xo)
    assert _anorm_rel(Ad, x, xo) <= max(1e-10, 2 * spread)
    r_gpu = np.linalg.norm(b - Ad @ x)
    r_orc = np.linalg.norm(b - Ad @ xo)
    assert abs(r_gpu - r_orc) <= 1e-12 * np.linalg.norm(b)
    assert abs(rep["rnorm"] - r_gpu) <= 1e-9 * np.linalg.norm(b)
    assert rep["istop"] in (1, 2) and rep["cond_est"] < 10


@pytest.mark.parametrize("case", ["cfg1", "ragged_rfm"])
@pytest.mark.parametrize("prec", ["f64", "f64emu"])
def test_restarted_solve_matches_oracle(csls, case, prec):
    """One LSQR restart from the solution found (the correction from r = b - A x): the GPU's restarted
    solution equals the oracle's restarted one in the A-norm to 1e-10, and both are at least as close
    to the dense Householder solution as the first solves are."""
    p = SKETCH_CASES[case]()
    Ad = p.dense()
    b = p.b[0]
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=11, prec=prec)
    x1, rep1 = csls.csls_solve(F, A, torch.tensor(b, device="cuda"))
    x, rep = csls.csls_solve(F, A, torch.tensor(b, device="cuda"), refine=1)
    x1, x = x1.cpu().numpy(), x.cpu().numpy()
    assert rep["iterations_refine"] > 0 and rep["iterations"] == rep1["iterations"] + rep["iterations_refine"]
    _, xo, info = oracle.csqrp_lsqr(p, b, seed=11, refine=1)
    assert info["iterations_refine"] > 0
    x_hh, _ = oracle.hhqr_solve(Ad, b)
    assert _anorm_rel(Ad, x, xo) <= 1e-10
    assert _anorm_rel(Ad, x, x_hh) <= max(2e-12, 2 * _anorm_rel(Ad, x1, x_hh))
    assert abs(rep["rnorm"] - np.linalg.norm(b - Ad @ x)) <= 1e-9 * np.linalg.norm(b)


def test_restart_removes_the_sketch_dependence(csls):
    """On a 3x3-box RFM system (cond(A) ~ 1e9) the first solves with two different sketches end
    ~1e-10 apart in the A-norm (the implicit form's rounding floor moves with R); after one restart
    they agree to 1e-12 and sit within 1e-11 of the dense Householder solution."""
    p = poisson2d(3, 3, 150, 25, 25, R=2.0, seed=2)     # 6,525 x 1,350
    Ad = p.dense()
    b = p.b[0]
    A = dev(csls, p)
    xs = []
    for seed in (1, 2):
        F = csls.csls_factor(A, seed=seed, prec="f64emu")
        x, rep = csls.csls_solve(F, A, torch.tensor(b, device="cuda"), refine=1)
        xs.append(x.cpu().numpy())
    x_hh, _ = oracle.hhqr_solve(Ad, b)
    assert _anorm_rel(Ad, xs[0], xs[1]) <= 1e-12
    for x in xs:
        assert _anorm_rel(Ad, x, x_hh) <= 1e-11


def test_fixed_iterations_track_oracle(csls):
    """Early iterates match the oracle's when both preconditioners agree to
    rounding (a well-conditioned sketch; on the RFM sketches the two R factors
    differ by ~cond(SA) 2^-53, which already moves the early iterates)."""
    rng = np.random.default_rng(26)
    A = random_sparse(3000, 150, 10, rng, scale_exp=3.0)
    b = rng.standard_normal(3000)
    F = csls.csls_factor(dev(csls, A), s=600, seed=5)
    fac = oracle.factor(A, 600, 5)
    for k in (1, 2, 4, 8):
        x, rep = csls.csls_solve(F, dev(csls, A), torch.tensor(b, device="cuda"), fixed_iters=k)
        xo, info = oracle.lsqr(A, b, fac["R"], "qr", fixed_iters=k)
        assert rep["iterations"] == k
        assert _rel(x.cpu().numpy(), xo) < 1e-10


def test_multi_rhs_block_matches_single_and_oracle(csls):
    """The block form (independent recurrences sharing the passes over A and R)
    gives each column the single-right-hand-side result up to rounding, and
    matches the oracle; 19 columns exercise a ragged last group of 8."""
    modes = tuple((a, c) for a in range(1, 6) for c in range(1, 5))[:19]
    p = poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7, modes=modes)
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=3)
    B = torch.tensor(p.b, device="cuda")
    X, rep = csls.csls_solve(F, A, B)
    assert X.shape == (19, p.n)
    Ad = p.dense()
    fac = oracle.factor(p, min(4 * p.n, p.m), 3)
    for k in (0, 7, 8, 18):
        xk, repk = csls.csls_solve(F, A, B[k])
        assert _anorm_rel(Ad, X[k].cpu().numpy(), xk.cpu().numpy()) < 1e-12
        xo, info = oracle.lsqr(p, p.b[k], fac["R"], "qr")
        x_hh, _ = oracle.hhqr_solve(Ad, p.b[k])
        assert _anorm_rel(Ad, X[k].cpu().numpy(), xo) <= max(1e-10, 2 * _anorm_rel(Ad, x_hh, xo))
    assert rep["iterations"] >= repk["iterations"]


def test_multi_rhs_block_restart_matches_oracle_restart(csls):
    """Block LSQR with one restart (tol 1e-8, the bench's rule) against the oracle's restarted CSQRP-LSQR
    of the same sketch, the dense solve and the restarted single-right-hand-side GPU solve. This RFM system
    is far from consistent (||r|| / ||b|| ~ 1e-2), so at tol 1e-8 rule S2 leaves the oracle itself ~2e-10
    from the dense solve: the bar is max(1e-10, twice that distance)."""
    modes = tuple((a, c) for a in range(1, 6) for c in range(1, 5))[:11]
    p = poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7, modes=modes)
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=3)
    B = torch.tensor(p.b, device="cuda")
    X, rep = csls.csls_solve(F, A, B, tol=1e-8, refine=1)
    assert rep["status"] == 0 and rep["iterations_refine"] > 0
    Ad = p.dense()
    for k in (0, 5, 10):
        _, xo, _ = oracle.csqrp_lsqr(p, p.b[k], seed=3, tol=1e-8, refine=1)
        x_hh, _ = oracle.hhqr_solve(Ad, p.b[k])
        xg = X[k].cpu().numpy()
        bar = max(1e-10, 2 * _anorm_rel(Ad, xo, x_hh))   # the problem's own spread at this tolerance
        assert _anorm_rel(Ad, xg, xo) <= bar
        assert _anorm_rel(Ad, xg, x_hh) <= bar
        xk, _ = csls.csls_solve(F, A, B[k], tol=1e-8, refine=1)
        assert _anorm_rel(Ad, xg, xk.cpu().numpy()) <= bar


def test_multi_rhs_fixed_iterations_track_single(csls):
    rng = np.random.default_rng(27)
    A = random_sparse(3000, 150, 10, rng, scale_exp=3.0)
    Bn = rng.standard_normal((10, 3000))
    F = csls.csls_factor(dev(csls, A), s=600, seed=5)
    B = torch.tensor(Bn, device="cuda")
    X, rep = csls.csls_solve(F, dev(csls, A), B, fixed_iters=6)
    fac = oracle.factor(A, 600, 5)
    for k in range(10):
        xo, _ = oracle.lsqr(A, Bn[k], fac["R"], "qr", fixed_iters=6)
        assert _rel(X[k].cpu().numpy(), xo) < 1e-10


def test_multi_rhs_block_pieces_track_oracle(csls):
    """n = 4,800: R has 75 diagonal blocks, so the block triangular solves hand each step's products with
    solutions more than 32 steps old to worker CTAs (up to three pieces a step, summed in piece order).
    Twelve right-hand sides (a half-empty second group of 8): after 8 fixed iterations each column matches
    the oracle's LSQR run with the same R to 1e-10, and the tol-plus-restart solutions match the single
    right-hand-side solves in the A-norm to 1e-10."""
    rng = np.random.default_rng(31)
    A = random_sparse(20000, 4800, 10, rng, scale_exp=3.0)
    assert (A.n + 63) // 64 > 2 * 32 + 1
    Bn = rng.standard_normal((12, 20000))
    Ag = dev(csls, A)
    F = csls.csls_factor(Ag, seed=5)
    R = F.R().cpu().numpy()
    B = torch.tensor(Bn, device="cuda")
    X, rep = csls.csls_solve(F, Ag, B, fixed_iters=8)
    assert rep["iterations"] == 8
    for k in (0, 7, 8, 11):
        xo, _ = oracle.lsqr(A, Bn[k], R, "qr", fixed_iters=8)
        assert _rel(X[k].cpu().numpy(), xo) < 1e-10
    X2, rep2 = csls.csls_solve(F, Ag, B, tol=1e-8, refine=1)
    assert rep2["status"] == 0
    for k in (0, 9):
        xk, _ = csls.csls_solve(F, Ag, B[k], tol=1e-8, refine=1)
        xb, xs = X2[k].cpu().numpy(), xk.cpu().numpy()
        assert np.linalg.norm(oracle.spmv(A, xb - xs)) <= 1e-10 * np.linalg.norm(oracle.spmv(A, xs))


def test_svd_variant_rank_deficient(csls):
    rng = np.random.default_rng(24)
    base = random_sparse(900, 40, 6, rng).dense()
    Ad = np.concatenate([base, base[:, :5] @ rng.standard_normal((5, 6))], axis=1)   # rank 40 of 46
    b = rng.standard_normal(900)
    A = csr_from_dense(Ad)
    F = csls.csls_factor(dev(csls, A), s=184, seed=2, variant="svd")
    x, rep = csls.csls_solve(F, dev(csls, A), torch.tensor(b, device="cuda"), variant="svd", tol=1e-14, maxit=200)
    assert rep["r"] == 40
    x_mn = np.linalg.lstsq(Ad, b, rcond=None)[0]
    assert _rel(x.cpu().numpy(), x_mn) < 1e-9
    fac, xo, _ = oracle.csqrp_lsqr(A, b, s=184, seed=2, variant="svd", tol=1e-14, maxit=200)
    assert fac["r"] == 40 and _rel(x.cpu().numpy(), xo) < 1e-9


def test_svd_variant_full_rank_cfg1(csls):
    p = config_problem("cfg1")
    b = p.b[0]
    F = csls.csls_factor(dev(csls, p), seed=11, variant="svd")
    x, rep = csls.csls_solve(F, dev(csls, p), torch.tensor(b, device="cuda"), variant="svd")
    fac, xo, _ = oracle.csqrp_lsqr(p, b, seed=11, variant="svd")
    Ad = p.dense()
    x_hh, _ = oracle.hhqr_solve(Ad, b)
    assert rep["r"] == fac["r"]
    assert _anorm_rel(Ad, x.cpu().numpy(), xo) <= max(1e-10, 2 * _anorm_rel(Ad, x_hh, xo))


def test_backward_matches_oracle_adjoint(csls):
    prob = scaled_random_sparse(1000, 100, per_row=10, cond_exp=4.0, seed=5)
    A = CSR(prob.m, prob.n, prob.row_ptr, prob.col, prob.val)
    b = prob.b[0]
    Ag = dev(csls, prob)
    F = csls.csls_factor(Ag, seed=8)
    bt = torch.tensor(b, device="cuda")
    x, _ = csls.csls_solve(F, Ag, bt, tol=1e-14, maxit=300)
    gx = 2.0 * (x - torch.tensor(prob.x_true, device="cuda"))
    gb, gv, rep = csls.csls_solve_backward(F, Ag, bt, x, gx, tol=1e-14, maxit=300)
    x_hh, RA = oracle.hhqr_solve(A.dense(), b)
    lam, gbo, gvo = oracle.adjoint(A, b, x.cpu().numpy(), RA, gx.cpu().numpy())
    assert _rel(gb.cpu().numpy(), gbo) < 1e-9
    assert _rel(gv.cpu().numpy(), gvo) < 1e-9


def test_autograd_function(csls):
    prob = scaled_random_sparse(600, 40, per_row=6, cond_exp=2.0, seed=9)
    A = dev(csls, prob)
    val = A.val.clone().requires_grad_(True)
    b = torch.tensor(prob.b[0], device="cuda", requires_grad=True)
    x = csls.CslsSolve.apply(val, b, A.row_ptr, A.col, A.m, A.n, dict(tol=1e-14, maxit=200))
    loss = ((x - torch.tensor(prob.x_true, device="cuda")) ** 2).sum()
    loss.backward()
    Ad = CSR(prob.m, prob.n, prob.row_ptr, prob.col, prob.val)
    x_hh, RA = oracle.hhqr_solve(Ad.dense(), prob.b[0])
    _, gbo, gvo = oracle.adjoint(Ad, prob.b[0], x.detach().cpu().numpy(), RA,
                                 2.0 * (x.detach().cpu().numpy() - prob.x_true))
    assert _rel(b.grad.cpu().numpy(), gbo) < 1e-9
    assert _rel(val.grad.cpu().numpy(), gvo) < 1e-9


# ----------------------------------------------------------------------------- status codes

def test_nonfinite_rhs(csls):
    p = config_problem("cfg1")
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=1)
    b = torch.tensor(p.b[0], device="cuda")
    b[17] = float("nan")
    x, rep = csls.csls_solve(F, A, b, raise_on_error=False)
    assert rep["status"] == 5


def test_nonfinite_matrix(csls):
    p = config_problem("cfg1")
    val = p.val.copy()
    val[123] = np.inf
    A = csls.Csr.from_numpy(p.row_ptr, p.col, val, p.m, p.n)
    with pytest.raises(csls.CslsError) as e:
        csls.csls_factor(A, seed=1)
    assert e.value.status == 5


def test_rank_deficient_qr(csls):
    rng = np.random.default_rng(25)
    Ad = random_sparse(500, 20, 5, rng).dense()
    Ad[:, 7] = 0.0   # a zero column: R(7, 7) = 0
    with pytest.raises(csls.CslsError) as e:
        csls.csls_factor(dev(csls, csr_from_dense(Ad)), s=80, seed=1)
    assert e.value.status == 2


def test_not_converged(csls):
    p = config_problem("cfg1")
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=1)
    x, rep = csls.csls_solve(F, A, torch.tensor(p.b[0], device="cuda"), maxit=2, raise_on_error=False)
    assert rep["status"] == 3 and rep["iterations"] == 2


def test_bounded_wait_timeout_then_recovery(csls):
    """spin_limit 0 makes every grid-barrier wait give up at once: the factor
    returns CSLS_ERR_TIMEOUT instead of hanging, and the context stays usable."""
    p = config_problem("cfg1")
    A = dev(csls, p)
    with pytest.raises(csls.CslsError) as e:
        csls.csls_factor(A, seed=1, spin_limit=0)
    assert e.value.status == 7
    F = csls.csls_factor(A, seed=1)
    x, rep = csls.csls_solve(F, A, torch.tensor(p.b[0], device="cuda"))
    assert rep["status"] == 0


def test_f32_factor_guard(csls):
    p = config_problem("cfg1")
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=11, prec="f32")
    x, rep = csls.csls_solve(F, A, torch.tensor(p.b[0], device="cuda"), prec="f32", raise_on_error=False)
    assert rep["status"] in (0, 6)
    assert (rep["status"] == 6) == (rep["cond_est"] >= 10)
    if rep["status"] == 0:
        Ad = p.dense()
        _, xo, _ = oracle.csqrp_lsqr(p, p.b[0], seed=11)
        x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
        assert _anorm_rel(Ad, x.cpu().numpy(), xo) <= max(1e-9, 4 * _anorm_rel(Ad, x_hh, xo))
    rep2 = csls.csls_solve(F, A, torch.tensor(p.b[0], device="cuda"), guard_cond=1.0001, raise_on_error=False)[1]
    assert rep2["status"] == 6
    # the guard fires at the first checkpoint (32 iterations, polled every check_every)
    assert rep2["iterations"] <= 48 and rep2["cond_est"] >= 1.0001


def test_batch_f32_guard_per_instance(csls):
    from workloads import batched_instances
    probs = batched_instances(count=3)
    As = [dev(csls, p) for p in probs]
    Fs = [csls.csls_factor(As[0], seed=4), csls.csls_factor(As[1], seed=4, prec="f32"),
          csls.csls_factor(As[2], seed=4)]
    bs = [torch.tensor(p.b[0], device="cuda") for p in probs]
    xs, reps, status = csls.csls_batch_solve(Fs, As, bs, guard_cond=1.0001, raise_on_error=False)
    assert status == 6 and [r["status"] for r in reps] == [0, 6, 0]
    assert reps[1]["iterations"] == 32 and reps[1]["cond_est"] >= 1.0001
    for k in (0, 2):
        x1, rep1 = csls.csls_solve(Fs[k], As[k], bs[k])
        assert abs(reps[k]["iterations"] - rep1["iterations"]) <= max(2, rep1["iterations"] // 20)
        # s = min(4n, m): where m < 4n the sketch embeds less well and cond(A M) may pass 10
        assert abs(reps[k]["cond_est"] - rep1["cond_est"]) <= 0.05 * rep1["cond_est"]


# ----------------------------------------------------------------------------- emulated FP64 trailing updates

def test_emulated_factor_matches_oracle_well_conditioned(csls):
    rng = np.random.default_rng(21)
    A = random_sparse(3000, 200, 12, rng)   # 7 panels (ragged), several row chunks
    Re = csls.csls_factor(dev(csls, A), s=800, seed=9, prec="f64emu").R().cpu().numpy()
    Ro = oracle.factor(A, 800, 9)["R"]
    assert _rel(Re, Ro) < 1e-10
    assert np.all(np.diag(Re) >= 0) and np.all(np.tril(Re, -1) == 0)


@pytest.mark.parametrize("m,n,s", [(1001, 300, 1001), (3000, 200, 799)])
def test_emulated_factor_odd_sketch_height(csls, m, n, s):
    # an odd number of sketch rows: the last 128-row tile of every trailing update runs past s, and
    # 64-column outer blocks leave ragged 32-column tiles
    rng = np.random.default_rng(m + n)
    A = random_sparse(m, n, 12, rng)
    R = csls.csls_factor(dev(csls, A), s=s, seed=13, prec="f64emu").R().cpu().numpy()
    h, d = oracle.hash_rows(m, s, 13)
    SA = oracle.sketch(A, s, h, d)
    assert np.linalg.norm(R.T @ R - SA.T @ SA) / np.linalg.norm(SA) ** 2 < 1e-11
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)


@pytest.mark.parametrize("m,n,s", [(2000, 130, 130), (700, 192, 200)])
def test_emulated_factor_short_outer_blocks(csls, m, n, s):
    # s at or just above n: the last outer blocks have L <= 64 rows below their first column, so the
    # panel's CTA that holds the block's diagonal rows holds every row (and the grid shrinks to two
    # CTAs), or the rows past the diagonal ones fill one short chunk
    rng = np.random.default_rng(7 * m + n)
    A = random_sparse(m, n, 12, rng)
    R = csls.csls_factor(dev(csls, A), s=s, seed=17, prec="f64emu").R().cpu().numpy()
    h, d = oracle.hash_rows(m, s, 17)
    SA = oracle.sketch(A, s, h, d)
    assert np.linalg.norm(R.T @ R - SA.T @ SA) / np.linalg.norm(SA) ** 2 < 1e-11
    assert np.all(np.diag(R) >= 0) and np.all(np.tril(R, -1) == 0)
    # R itself moves by up to cond(SA) x the backward error (cond 2.4e3 and 1.9e2 here)
    Ro = oracle.factor(A, s, 17)["R"]
    assert _rel(R, Ro) < 1e-8


@pytest.mark.parametrize("case", ["cfg1", "ragged_rfm"])
def test_emulated_factor_rfm_backward_error_and_solve(csls, case):
    p = SKETCH_CASES[case]()
    s = min(4 * p.n, p.m)
    F = csls.csls_factor(dev(csls, p), seed=11, prec="f64emu")
    R = F.R().cpu().numpy()
    h, d = oracle.hash_rows(p.m, s, 11)
    SA = oracle.sketch(p, s, h, d)
    err = np.linalg.norm(R.T @ R - SA.T @ SA) / np.linalg.norm(SA) ** 2
    assert err < 1e-11
    b = p.b[0]
    x, rep = csls.csls_solve(F, dev(csls, p), torch.tensor(b, device="cuda"))
    Ad = p.dense()
    _, xo, _ = oracle.csqrp_lsqr(p, b, seed=11)
    x_hh, _ = oracle.hhqr_solve(Ad, b)
    assert _anorm_rel(Ad, x.cpu().numpy(), xo) <= max(1e-10, 2 * _anorm_rel(Ad, x_hh, xo))
    assert rep["istop"] in (1, 2) and rep["cond_est"] < 10


# ----------------------------------------------------------------------------- ragged batch in one graph launch

def test_batch_solve_uneven_instances(csls, tmp_path):
    from workloads import batched_instances
    probs = batched_instances(count=7)           # grids 2..6, J in {50, 100, 150}, uneven point counts
    As = [dev(csls, p) for p in probs]
    Fs = [csls.csls_factor(A, seed=2 + k) for k, A in enumerate(As)]
    cache = str(tmp_path / "tune.json")
    groups = [csls.csls_autotune(F, A, cache=cache) for F, A in zip(Fs, As)]
    assert all(g in (4, 8, 16, 32) and gt in (4, 8, 16, 32) for g, gt in groups)
    assert csls.csls_autotune(Fs[0], As[0], cache=cache) == groups[0]   # served from the cache
    bs = [torch.tensor(p.b[0], device="cuda") for p in probs]
    xs, reps, status = csls.csls_batch_solve(Fs, As, bs)
    assert status == 0
    for k, p in enumerate(probs):
        # the batch kernels sum in another order than the single solve: the two agree to the
        # problem's own floating-point sensitivity, measured as the spread between two single
        # solves whose sketches differ (cond(A) ~ 1e9 here, so that spread is ~1e-10)
        x1, rep1 = csls.csls_solve(Fs[k], As[k], bs[k])
        x2, _ = csls.csls_solve(csls.csls_factor(As[k], seed=99 + k), As[k], bs[k])
        x1, x2, xb = (t.cpu().numpy() for t in (x1, x2, xs[k]))
        ax1 = np.linalg.norm(oracle.spmv(p, x1))
        spread = np.linalg.norm(oracle.spmv(p, x2 - x1)) / ax1
        assert np.linalg.norm(oracle.spmv(p, xb - x1)) / ax1 <= max(1e-10, 4 * spread), (k, spread)
        assert abs(reps[k]["iterations"] - rep1["iterations"]) <= max(2, rep1["iterations"] // 20)
        assert reps[k]["istop"] in (1, 2)
        if p.n <= 1800:
            Ad = p.dense()
            _, xo, _ = oracle.csqrp_lsqr(p, p.b[0], s=min(4 * p.n, p.m), seed=2 + k)
            x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
            assert _anorm_rel(Ad, xb, xo) <= max(1e-10, 2 * _anorm_rel(Ad, x_hh, xo))


# ----------------------------------------------------------------------------- warm start (Remark 3.1)

@pytest.mark.parametrize("prec", ["f64", "f64emu"])
def test_warm_start_point_and_solve_match_oracle(csls, prec):
    p = SKETCH_CASES["cfg1"]()
    A = dev(csls, p)
    b = torch.tensor(p.b[0], device="cuda")
    s = min(4 * p.n, p.m)
    F, x0 = csls.csls_factor_warm(A, b, seed=11, prec=prec)
    # x0 = argmin ||S (A x - b)||: compared in the sketched norm, the one the sketched problem fixes
    x0o, Sb = oracle.sketch_solve(p, p.b[0], s, seed=11)
    h, d = oracle.hash_rows(p.m, s, 11)
    SA = oracle.sketch(p, s, h, d)
    x0g = x0.cpu().numpy()
    assert np.linalg.norm(SA @ (x0g - x0o)) <= 1e-10 * np.linalg.norm(SA @ x0o)
    # LSQR from x0: same solution as the cold start and the oracle's warm run, in fewer iterations
    xw, repw = csls.csls_solve(F, A, b, x=x0.clone(), warm_start=1)
    xc, repc = csls.csls_solve(F, A, b)
    _, xo, io = oracle.csqrp_lsqr(p, p.b[0], seed=11, warm=True)
    _, xoc, _ = oracle.csqrp_lsqr(p, p.b[0], seed=11)
    Ad = p.dense()
    x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
    # reading R2: solutions that meet the 1e-12 stopping rule lie within the O1-O2 spread of each
    # other; the warm oracle run may land much closer to O1 than the cold one, so the spread is
    # taken over both oracle runs
    spread = max(_anorm_rel(Ad, x_hh, xo), _anorm_rel(Ad, x_hh, xoc))
    assert _anorm_rel(Ad, xw.cpu().numpy(), xo) <= max(1e-10, 2 * spread)
    assert _anorm_rel(Ad, xw.cpu().numpy(), xc.cpu().numpy()) <= max(1e-10, 2 * spread)
    assert repw["iterations"] < repc["iterations"]
    assert abs(repw["iterations"] - io["iterations"]) <= 3
    assert abs(repw["bnorm"] - np.linalg.norm(p.b[0])) <= 1e-12 * np.linalg.norm(p.b[0])
    assert repw["istop"] in (1, 2) and repw["cond_est"] < 10


def test_warm_start_well_conditioned_exact_parity(csls):
    rng = np.random.default_rng(31)
    Acpu = random_sparse(3000, 120, 8, rng)
    b = rng.standard_normal(3000)
    A = dev(csls, Acpu)
    F, x0 = csls.csls_factor_warm(A, torch.tensor(b, device="cuda"), s=480, seed=4)
    x0o, _ = oracle.sketch_solve(Acpu, b, 480, seed=4)
    assert _rel(x0.cpu().numpy(), x0o) < 1e-11
    fac = oracle.factor(Acpu, 480, 4)
    for k in (1, 3, 6):
        xk, _ = csls.csls_solve(F, A, torch.tensor(b, device="cuda"), x=x0.clone(), warm_start=1, fixed_iters=k)
        xo, _ = oracle.lsqr(Acpu, b, fac["R"], "qr", fixed_iters=k, x0=x0o)
        assert _rel(xk.cpu().numpy(), xo) < 1e-10
    # several right-hand sides, each from its own starting point, equal the one-by-one solves
    B = torch.tensor(np.stack([b, 2 * b + 1]), device="cuda")
    X0 = torch.stack([x0, 2 * x0])
    X, _ = csls.csls_solve(F, A, B, x=X0.clone(), warm_start=1)
    for k in range(2):
        xk, _ = csls.csls_solve(F, A, B[k], x=X0[k].clone(), warm_start=1)
        assert torch.equal(X[k], xk)


def test_warm_start_argument_errors(csls):
    p = SKETCH_CASES["cfg1"]()
    A = dev(csls, p)
    b = torch.tensor(p.b[0], device="cuda")
    with pytest.raises(csls.CslsError) as e:
        csls.csls_factor_warm(A, b, seed=1, variant="svd")
    assert e.value.status == 1
    F = csls.csls_factor(A, seed=1)
    _, _, st = csls.csls_batch_solve([F], [A], [b], warm_start=1, raise_on_error=False)
    assert st == 1


# ----------------------------------------------------------------------------- explicit form (Algorithm 1 steps 4-6)

def test_explicit_form_well_conditioned_matches_oracle(csls):
    rng = np.random.default_rng(41)
    Acpu = random_sparse(2500, 150, 8, rng)   # 3 diagonal blocks (ragged), 40 row tiles (ragged)
    b = rng.standard_normal(2500)
    A = dev(csls, Acpu)
    F = csls.csls_factor(A, s=600, seed=6)
    B = csls.csls_form_b(F, A).cpu().numpy().T
    fac = oracle.factor(Acpu, 600, 6)
    Bo = oracle.form_b(Acpu, fac)
    assert _rel(B, Bo) < 1e-10
    for k in (1, 4):
        x, _ = csls.csls_solve_explicit(F, torch.tensor(B.T.copy(), device="cuda"), torch.tensor(b, device="cuda"),
                                        fixed_iters=k)
        xo, _, _ = oracle.explicit_lsqr(Acpu, b, fac, fixed_iters=k)
        assert _rel(x.cpu().numpy(), xo) < 1e-10


def test_explicit_form_rfm(csls):
    p = SKETCH_CASES["cfg1"]()
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=11)
    Bt = csls.csls_form_b(F, A)
    B = Bt.cpu().numpy().T
    Ad = p.dense()
    R = F.R().cpu().numpy()
    assert np.linalg.norm(B @ R - Ad) <= 1e-12 * np.linalg.norm(Ad)   # B R = A with this factor's R
    sv = np.linalg.svd(B, compute_uv=False)
    assert sv[0] / sv[-1] < 10                                          # Theorem 3.2
    x, rep = csls.csls_solve_explicit(F, Bt, torch.tensor(p.b[0], device="cuda"))
    fac = oracle.factor(p, 4 * p.n, 11)
    xo, _, _ = oracle.explicit_lsqr(p, p.b[0], fac)
    x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
    _, xi, _ = oracle.csqrp_lsqr(p, p.b[0], seed=11)
    spread = max(_anorm_rel(Ad, x_hh, xo), _anorm_rel(Ad, x_hh, xi))
    assert _anorm_rel(Ad, x.cpu().numpy(), xo) <= max(1e-10, 2 * spread)
    assert rep["istop"] in (1, 2) and rep["cond_est"] < 10


def test_explicit_form_svd_rank_deficient(csls):
    from workloads import table_c1_problem
    p = table_c1_problem("rel6")
    A = dev(csls, p)
    F = csls.csls_factor(A, seed=3, variant="svd")
    Bt = csls.csls_form_b(F, A)
    assert Bt.shape[0] == p.info["rank"]
    x, rep = csls.csls_solve_explicit(F, Bt, torch.tensor(p.b[0], device="cuda"), tol=1e-14, maxit=500)
    Ad = p.dense()
    x_mn = np.linalg.lstsq(Ad, p.b[0], rcond=None)[0]
    assert np.linalg.norm(x.cpu().numpy() - x_mn) <= 1e-8 * np.linalg.norm(x_mn)
    assert rep["cond_est"] < 10


# ----------------------------------------------------------------------------- RFM assembly on the device

def _assemble_on_device(csls, p):
    from workloads import rfm_row_descriptors
    rows = rfm_row_descriptors(p)
    rows_dev = torch.from_numpy(rows.view(np.uint8).copy()).cuda()
    k = torch.tensor(p.k, device="cuda")
    c = torch.tensor(p.c, device="cuda")
    r_half = 0.5 / np.asarray(p.grid, dtype=np.float64)
    return csls.csls_rfm_assemble(p.dim, r_half, p.J, k, c, rows_dev)


@pytest.mark.parametrize("case", ["cfg1", "ragged2d", "box3d"])
def test_rfm_assembly_matches_generator(csls, case):
    from workloads import poisson3d
    p = {"cfg1": lambda: config_problem("cfg1"),
         "ragged2d": lambda: poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7),
         "box3d": lambda: poisson3d(2, 3, 2, 24, 5, e_bc=4, e_if=3, R=1.0, seed=9)}[case]()
    A = _assemble_on_device(csls, p)
    assert (A.m, A.n, A.nnz) == (p.m, p.n, p.nnz)
    assert np.array_equal(A.row_ptr.cpu().numpy(), p.row_ptr)
    assert np.array_equal(A.col.cpu().numpy(), p.col)
    v = A.val.cpu().numpy()
    assert np.all(np.abs(v - p.val) <= 1e-13 * np.maximum(1.0, np.abs(p.val)))
    # the device-assembled matrix gives the same least-squares solution
    b = torch.tensor(p.b[0], device="cuda")
    x1, _ = csls.csls_solve(csls.csls_factor(A, seed=3), A, b)
    Ah = dev(csls, p)
    x2, _ = csls.csls_solve(csls.csls_factor(Ah, seed=3), Ah, b)
    Ad = p.dense()
    assert _anorm_rel(Ad, x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-9


def test_rfm_assembly_argument_errors(csls):
    p = config_problem("cfg1")
    from workloads import rfm_row_descriptors
    rows = torch.from_numpy(rfm_row_descriptors(p).view(np.uint8).copy()).cuda()
    k = torch.tensor(p.k, device="cuda")
    c = torch.tensor(p.c, device="cuda")
    with pytest.raises(csls.CslsError):
        csls.csls_rfm_assemble(2, [0.25, -1.0], p.J, k, c, rows)


@pytest.mark.parametrize("count", [0, 1, 7, 1 << 20, (1 << 20) + 3])
def test_read_probe_checksum(csls, count):
    """The streaming-read probe touches every word exactly once: its per-CTA partials sum (mod 2^64)
    to the wrap-around sum of the buffer's 64-bit words, for every launch shape it accepts."""
    rng = np.random.default_rng(count)
    words = rng.integers(0, 2 ** 63, size=count, dtype=np.int64).view(np.uint64)
    expect = int(np.sum(words, dtype=np.uint64))
    buf = torch.from_numpy(words.view(np.int64).copy()).cuda()
    for ctas, unroll in ((1, 1), (2, 8), (4, 4), (3, 2)):
        part = csls.csls_read_probe(buf, ctas, unroll).cpu().numpy().view(np.uint64)
        assert int(np.sum(part, dtype=np.uint64)) == expect


def test_read_probe_argument_errors(csls):
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(csls.CslsError):
        csls.csls_read_probe(buf, 5, 8)
    with pytest.raises(csls.CslsError):
        csls.csls_read_probe(buf, 2, 3)
    with pytest.raises(csls.CslsError):   # 8-byte offset: not 16-byte aligned
        csls.csls_read_probe(buf[1:], 2, 8)


@pytest.mark.parametrize("n", [40, 150, 333, 2600, 9700])
@pytest.mark.parametrize("prec", ["f64", "f64emu"])
def test_precond_apply_chain_lengths(csls, n, prec):
    """Both triangular solves with a binary64 R against the oracle's substitutions, over chain lengths
    from one 64-row block to more blocks than an SM count (workers that start only after earlier
    ones finish), with ragged last blocks; repeated launches give identical bits."""
    rng = np.random.default_rng(n)
    m = 3 * n + 17
    A = random_sparse(m, n, 8, rng, scale_exp=3.0)
    Ad = dev(csls, A)
    F = csls.csls_factor(Ad, seed=5, prec=prec)
    R = F.R().cpu().numpy()
    v = rng.standard_normal(n)
    vt = torch.tensor(v, device="cuda")
    z = csls.csls_precond_apply(F, vt)
    zt = csls.csls_precond_apply(F, vt, trans=True)
    assert _rel(z.cpu().numpy(), oracle.trsv_upper(R, v)) < 1e-12
    assert _rel(zt.cpu().numpy(), oracle.trsv_upper_trans(R, v)) < 1e-12
    assert torch.equal(csls.csls_precond_apply(F, vt), z)
    assert torch.equal(csls.csls_precond_apply(F, vt, trans=True), zt)


@pytest.mark.parametrize("prec", ["f64emu", "f64", "f32"])
def test_theorem_3_2_sweep_on_gpu(csls, prec):
    """Theorem 3.2 on the GPU factors: with cond(A) swept over 12 decades by column scaling, cond(A R^-1)
    (exact, from the dense B = A R^-1 with the GPU's R) stays below 10 and flat for the binary64 and
    emulated factors. For every factor, the solve's estimate (the extreme singular values of the
    Golub-Kahan bidiagonal it built) is a lower bound of that exact value, and the binary32 factor's guard
    rejects it exactly when the estimate reaches 10."""
    rng = np.random.default_rng(10)
    base = random_sparse(2000, 50, 6, rng)
    conds = []
    guard = {v: k for k, v in csls.STATUS_NAMES.items()}["CSLS_ERR_PRECOND_GUARD"]
    for p in (0, 4, 8, 12):
        A = CSR(base.m, base.n, base.row_ptr, base.col, base.val * (10.0 ** (-p * np.arange(50) / 49))[base.col])
        Ad = dev(csls, A)
        F = csls.csls_factor(Ad, s=200, seed=3, prec=prec)
        R = F.R().cpu().numpy().astype(np.float64)
        B = np.linalg.solve(R.T, A.dense().T).T
        c = float(np.linalg.cond(B))
        conds.append(c)
        b = torch.tensor(rng.standard_normal(base.m), device="cuda")
        _, rep = csls.csls_solve(F, Ad, b, tol=1e-12, raise_on_error=False, prec=prec)
        assert rep["cond_est"] <= c * (1 + 1e-3)
        if prec == "f32":
            assert rep["status"] == (guard if rep["cond_est"] >= 10 else 0)
        else:
            assert rep["status"] == 0
        if p >= 8:
            assert float(np.linalg.cond(A.dense())) > 1e6
    if prec != "f32":
        assert max(conds) < 10 and max(conds) / min(conds) < 1.5
    else:
        assert conds[0] < 10
