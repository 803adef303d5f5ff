"""Parity at the full workload sizes, in the launch configuration the benchmark
uses (binary64 sketch, emulated-FP64 trailing updates, tol 1e-12).

The oracle cannot run the whole method at these sizes, so it checks sampled
outputs it computes one by one and properties that hold at any size:
  * sketch: sampled rows of SA, bit for bit (the oracle sketches just the rows
    of A hashed to each sampled bucket, in ascending order);
  * factor: sampled entries of R^T R against (SA^T SA)_ij, with the two sketch
    columns recomputed by the oracle (backward error of the QR);
  * solve: the LSQR residual estimate against ||b - A x|| (oracle SpMV); the
    preconditioned condition estimate stays below 10 (Theorem 3.2); on the RFM
    workloads the computed coefficients reproduce the manufactured solution at
    held-out points (an error level fixed by the RFM space, far above solver
    error); on the column-scaled workload ||A (x - x_true)|| stays below the
    injected noise, as it must for the least-squares solution.
(A residual-optimality test ||A^T r|| / (||A|| ||r||) is not used: at cond(A) ~
1e10 the FP64 residual b - A x loses most of its digits to cancellation.)
"""
import numpy as np
import pytest
import torch

import oracle
from tests.helpers import CSR
from workloads import config_problem, scaled_random_sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csls():
    from paper_2409_15818_gb300 import build
    build.build()
    from paper_2409_15818_gb300 import csls as mod
    return mod


def _sub_rows(p, rows):
    rows = np.asarray(rows, dtype=np.int64)
    lens = p.row_ptr[rows + 1] - p.row_ptr[rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(p.row_ptr[r], p.row_ptr[r + 1]) for r in rows]) if len(rows) else np.zeros(0, int)
    return CSR(len(rows), p.n, rp, p.col[idx].copy(), p.val[idx].copy())


def _sub_cols(p, cols):
    """CSR of A(:, cols) (columns renumbered 0..len-1), same row order."""
    cols = np.asarray(cols)
    where = {c: k for k, c in enumerate(cols)}
    keep = np.isin(p.col, cols)
    rows = np.repeat(np.arange(p.m), np.diff(p.row_ptr))[keep]
    rp = np.zeros(p.m + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    newc = np.array([where[c] for c in p.col[keep]], dtype=np.int32)
    return CSR(p.m, len(cols), rp, newc, p.val[keep].copy())


def check_sketch_rows(csls, p, s, seed, nsample=48):
    A = csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)
    SA = csls.csls_sketch(A, s, seed)          # (n, s) storage of the column-major s x n sketch
    h, d = oracle.hash_rows(p.m, s, seed)
    rng = np.random.default_rng(seed)
    buckets = rng.choice(s, nsample, replace=False)
    for k in buckets:
        rows = np.nonzero(h == k)[0]            # ascending
        sub = _sub_rows(p, rows)
        want = oracle.sketch(sub, 1, np.zeros(len(rows), np.int32), d[rows])[0]
        got = SA[:, int(k)].cpu().numpy()
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), k
    del SA
    torch.cuda.empty_cache()


def check_factor_entries(F, p, s, seed, npairs=24):
    R = F.R()
    h, d = oracle.hash_rows(p.m, s, seed)
    rng = np.random.default_rng(seed + 1)
    n = p.n
    for _ in range(npairs):
        i, j = sorted(rng.choice(n, 2, replace=False))
        sub = _sub_cols(p, [i, j])
        SAij = oracle.sketch(sub, s, h, d)
        want = float(SAij[:, 0] @ SAij[:, 1])
        scale = float(np.linalg.norm(SAij[:, 0]) * np.linalg.norm(SAij[:, 1]))
        got = float(R[: i + 1, i] @ R[: i + 1, j])
        assert abs(got - want) <= 1e-11 * scale, (i, j, got, want)
        nii = float(R[: i + 1, i] @ R[: i + 1, i])
        assert abs(nii - float(SAij[:, 0] @ SAij[:, 0])) <= 1e-11 * float(SAij[:, 0] @ SAij[:, 0])
    diag = torch.diagonal(R)
    assert bool((diag > 0).all()) and bool((torch.tril(R, -1) == 0).all())


def check_solution(p, x, rep, b):
    x = x.cpu().numpy()
    r = b - oracle.spmv(p, x)
    rn = np.linalg.norm(r)
    assert abs(rep["rnorm"] - rn) <= 1e-8 * np.linalg.norm(b)
    assert rep["istop"] in (1, 2) and rep["cond_est"] < 10
    return x


def check_manufactured(p, x, tol):
    pts = np.random.default_rng(5).random((20000, p.dim))
    ue = p.exact(pts)
    err = np.linalg.norm(p.evaluate(x, pts) - ue) / np.linalg.norm(ue)
    assert err < tol, err
    return err


def test_cfg2_full_size(csls):
    p = config_problem("cfg2")
    s = 4 * p.n
    check_sketch_rows(csls, p, s, 1)
    A = csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)
    F = csls.csls_factor(A, seed=1, prec="f64emu")
    check_factor_entries(F, p, s, 1)
    b = p.b[0]
    x, rep = csls.csls_solve(F, A, torch.tensor(b, device="cuda"), tol=1e-12)
    xh = check_solution(p, x, rep, b)
    check_manufactured(p, xh, 1e-4)


def test_cfg5_full_size_f32_factor_passes_guard(csls):
    """Column-scaling ill-conditioning: the binary32 factor keeps cond(A R^-1) < 10."""
    p = config_problem("cfg5")
    A = csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)
    F = csls.csls_factor(A, seed=1, prec="f32")
    b = p.b[0]
    x, rep = csls.csls_solve(F, A, torch.tensor(b, device="cuda"), tol=1e-12)
    assert rep["status"] == 0
    xh = check_solution(p, x, rep, b)
    noise = np.linalg.norm(b - oracle.spmv(p, p.x_true))
    assert np.linalg.norm(oracle.spmv(p, xh - p.x_true)) <= 1.01 * noise
    del F
    torch.cuda.empty_cache()
    F64 = csls.csls_factor(A, seed=1, prec="f64emu")
    x64, rep64 = csls.csls_solve(F64, A, torch.tensor(b, device="cuda"), tol=1e-12)
    x64h = check_solution(p, x64, rep64, b)
    assert np.linalg.norm(oracle.spmv(p, x64h - p.x_true)) <= 1.01 * noise
    # the noise level is 1e-8, cond(A) ~ 1e10: both solutions fit the data equally well
    assert abs(rep["rnorm"] - rep64["rnorm"]) <= 1e-10 * np.linalg.norm(b)


def test_cfg3_full_size(csls):
    p = config_problem("cfg3")
    s = 4 * p.n
    check_sketch_rows(csls, p, s, 1, nsample=24)
    A = csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)
    F = csls.csls_factor(A, seed=1, prec="f64emu")
    check_factor_entries(F, p, s, 1, npairs=12)
    b = p.b[0]
    x, rep = csls.csls_solve(F, A, torch.tensor(b, device="cuda"), tol=1e-12)
    xh = check_solution(p, x, rep, b)
    check_manufactured(p, xh, 1e-2)


def test_backward_on_slice_at_ten_decades(csls):
    """The differentiated workload's own recipe on its 1,000 x 100 slice: 10 decades of column scaling,
    cond(A) ~ 1e10, L = ||x - x_true||^2.
      * Against the oracle's dense adjoint (lambda = R_A^-1 R_A^-T g from the Householder QR of A, at
        the GPU's x): dL/db to 1e-9; dL/d(values) to a bar set by the residual: r = b - A x is computed
        with |A||x| ~ 1 against |r| ~ 1e-8 (the injected noise), so its entries carry relative errors
        ~2^-53 / 1e-8; the bar is 10x the difference between two exact-arithmetic-equivalent dense
        evaluations of the gradient formula (the oracle's row loop and a dense product), at least 1e-9.
      * Against central differences of the GPU solve in b: L is quadratic in b, so a central
        difference is exact for any step and a step of 1 keeps the solve's own rounding (which the
        10 decades amplify) far below the difference. In the values L is not quadratic and the
        solve's rounding swamps any step small enough for the truncation error, so those are checked
        against the oracle only."""
    prob = scaled_random_sparse(1000, 100, per_row=10, cond_exp=10.0, seed=5)
    A = csls.Csr.from_numpy(prob.row_ptr, prob.col, prob.val, prob.m, prob.n)
    xt = torch.tensor(prob.x_true, device="cuda")
    opts = dict(seed=3, tol=1e-14, maxit=300, refine=1)
    F = csls.csls_factor(A, **opts)

    def loss(bb):
        x, _ = csls.csls_solve(F, A, bb, **opts)
        return float(((x - xt) ** 2).sum()), x

    b = torch.tensor(prob.b[0], device="cuda")
    L0, x = loss(b)
    gx = 2.0 * (x - xt)
    gb, gv, rep = csls.csls_solve_backward(F, A, b, x, gx, **opts)
    gb, gv = gb.cpu().numpy(), gv.cpu().numpy()
    Ad = prob.dense()
    xh = x.cpu().numpy()
    _, RA = oracle.hhqr_solve(Ad, prob.b[0])
    lam, gbo, gvo = oracle.adjoint(prob, prob.b[0], xh, RA, gx.cpu().numpy())
    rel = lambda a, r: float(np.linalg.norm(a - r) / np.linalg.norm(r))
    assert rel(gb, gbo) <= 1e-9
    rows = np.repeat(np.arange(prob.m), np.diff(prob.row_ptr))
    r_dense = prob.b[0] - Ad @ xh
    gv_dense = r_dense[rows] * lam[prob.col] - (Ad @ lam)[rows] * xh[prob.col]
    bar = max(1e-9, 10.0 * rel(gv_dense, gvo))
    assert rel(gv, gvo) <= bar, (rel(gv, gvo), bar)
    rng = np.random.default_rng(0)
    for i in rng.choice(prob.m, 12, replace=False):
        e = torch.zeros_like(b)
        e[int(i)] = 1.0
        fd = (loss(b + e)[0] - loss(b - e)[0]) / 2.0
        assert abs(fd - float(gb[int(i)])) <= 1e-6 * float(np.abs(gb).max())


def test_backward_finite_differences_on_slice(csls):
    """dL/db and dL/d(values) from the GPU adjoint against central differences of
    the GPU solve itself, on a 1,000 x 100 slice of the differentiated workload's
    recipe with 4 decades of column scaling (at the workload's 10 decades the
    solve's rounding swamps differences in the values; that case is checked
    against the oracle's dense adjoint and exact differences in b above)."""
    prob = scaled_random_sparse(1000, 100, per_row=10, cond_exp=4.0, seed=5)
    A = csls.Csr.from_numpy(prob.row_ptr, prob.col, prob.val, prob.m, prob.n)
    xt = torch.tensor(prob.x_true, device="cuda")
    opts = dict(seed=3, tol=1e-14, maxit=300)

    def loss(vals, bb):
        Ai = A.with_values(vals)
        F = csls.csls_factor(Ai, **opts)
        x, _ = csls.csls_solve(F, Ai, bb, **opts)
        return float(((x - xt) ** 2).sum()), x, F

    b = torch.tensor(prob.b[0], device="cuda")
    L0, x, F = loss(A.val, b)
    gb, gv, _ = csls.csls_solve_backward(F, A, b, x, 2.0 * (x - xt), **opts)
    rng = np.random.default_rng(0)
    h = 1e-6
    for i in rng.choice(prob.m, 12, replace=False):
        e = torch.zeros_like(b)
        e[int(i)] = h
        fd = (loss(A.val, b + e)[0] - loss(A.val, b - e)[0]) / (2 * h)
        assert abs(fd - float(gb[int(i)])) <= 1e-6 * float(gb.abs().max())
    for pidx in rng.choice(prob.nnz, 12, replace=False):
        # Richardson-extrapolated central differences (O(step^4) truncation) with a relative
        # step large enough that the forward solve's own accuracy does not dominate
        def central(step):
            e = torch.zeros_like(A.val)
            e[int(pidx)] = step
            return (loss(A.val + e, b)[0] - loss(A.val - e, b)[0]) / (2 * step)
        step = 1e-4 * abs(float(A.val[int(pidx)]))
        fd = (4.0 * central(step / 2) - central(step)) / 3.0
        assert abs(fd - float(gv[int(pidx)])) <= 1e-6 * float(gv.abs().max())
