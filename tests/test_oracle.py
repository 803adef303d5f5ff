"""Pins for the CPU oracle: each test ties one oracle function to something
other than itself -- a worked example from the paper, a closed form, a library
routine on a special case, brute force in exact rationals, or an invariant the
paper proves. Runs without a GPU."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg

import oracle
from tests.helpers import CSR, csr_from_dense, read_golden_rows, random_sparse
from workloads import config_problem, poisson2d, scaled_random_sparse


# ----------------------------------------------------------------------------- hash

def test_splitmix64_reference_sequence():
    want = [int(r[0], 16) for r in read_golden_rows("splitmix64_seed0.txt")[0]]
    got = [oracle.splitmix64_output(0, i) for i in range(3)]
    assert got == want


def test_hash_buckets_uniform_and_signs_balanced():
    m, s = 400_000, 997
    h, d = oracle.hash_rows(m, s, seed=12345)
    assert h.min() >= 0 and h.max() < s
    counts = np.bincount(h, minlength=s)
    expect = m / s
    chi2 = np.sum((counts - expect) ** 2 / expect)
    # chi-square with s-1 dof: mean s-1, sd sqrt(2(s-1)); allow 5 sd
    assert abs(chi2 - (s - 1)) < 5 * np.sqrt(2 * (s - 1))
    assert set(np.unique(d)) == {-1, 1}
    assert abs(d.astype(np.int64).sum()) < 5 * np.sqrt(m)
    # sign independent of bucket parity
    plus_even = np.mean(d[h % 2 == 0] == 1)
    assert abs(plus_even - 0.5) < 5 * 0.5 / np.sqrt(np.sum(h % 2 == 0))


# ----------------------------------------------------------------------------- sketch

def test_count_sketch_paper_example():
    S = np.array(read_golden_rows("count_sketch_example_s4_m5.txt")[0], dtype=np.float64)
    s, m = S.shape
    assert np.all(np.count_nonzero(S, axis=0) == 1)
    h = np.argmax(np.abs(S), axis=0).astype(np.int32)
    d = S[h, np.arange(m)].astype(np.int8)
    assert list(h + 1) == [2, 4, 1, 1, 3] and list(d) == [1, -1, -1, 1, 1]
    rng = np.random.default_rng(0)
    A = rng.integers(-9, 10, size=(m, 3)).astype(np.float64)
    got = oracle.sketch(csr_from_dense(A), s, h, d)
    np.testing.assert_array_equal(got, S @ A)


def test_sketch_bijective_is_signed_permutation():
    rng = np.random.default_rng(1)
    A = csr_from_dense(rng.standard_normal((40, 7)) * (rng.random((40, 7)) < 0.5))
    h = rng.permutation(40).astype(np.int32)
    d = rng.choice([-1, 1], 40).astype(np.int8)
    got = oracle.sketch(A, 40, h, d)
    want = np.zeros((40, 7))
    want[h] = d[:, None] * A.dense()
    np.testing.assert_array_equal(got, want)


def test_sketch_integer_matrix_exact_and_f32():
    rng = np.random.default_rng(2)
    Ad = rng.integers(-50, 51, size=(300, 20)).astype(np.float64) * (rng.random((300, 20)) < 0.3)
    A = csr_from_dense(Ad)
    h, d = oracle.hash_rows(300, 37, seed=7)
    S = np.zeros((37, 300))
    S[h, np.arange(300)] = d
    np.testing.assert_array_equal(oracle.sketch(A, 37, h, d), S @ Ad)
    np.testing.assert_array_equal(oracle.sketch(A, 37, h, d, np.float32), (S @ Ad).astype(np.float32))


# ----------------------------------------------------------------------------- QR

def test_qr_textbook_345():
    blocks = read_golden_rows("qr_345.txt")
    A = np.array(blocks[0], dtype=np.float64)
    R_want = np.array(blocks[1], dtype=np.float64)
    np.testing.assert_allclose(oracle.r_factor(A), R_want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("shape", [(300, 50), (97, 97), (64, 13)])
def test_qr_matches_lapack(shape):
    rng = np.random.default_rng(3)
    A = rng.standard_normal(shape)
    R = oracle.r_factor(A)
    Rl = np.linalg.qr(A, mode="r")
    Rl = Rl * np.sign(np.diag(Rl))[:, None]
    np.testing.assert_allclose(R, Rl, rtol=0, atol=1e-12 * np.abs(Rl).max())
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) >= 0)


def test_qr_backward_error_ill_conditioned():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((400, 60)) @ np.diag(10.0 ** -np.linspace(0, 12, 60))
    A = A @ np.linalg.qr(rng.standard_normal((60, 60)))[0]   # mix the scales
    R = oracle.r_factor(A)
    err = np.linalg.norm(R.T @ R - A.T @ A) / np.linalg.norm(A) ** 2
    assert err < 60 * 400 * np.finfo(float).eps


def test_qr_f32_close_to_f64():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((200, 40))
    R64 = oracle.r_factor(A)
    R32 = oracle.r_factor(A.astype(np.float32))
    assert np.abs(R32 - R64).max() < 50 * np.finfo(np.float32).eps * np.abs(R64).max()


# ----------------------------------------------------------------------------- TRSV, SpMV

def _frac_back_subst(R, v, upper_trans=False):
    n = len(v)
    Rf = [[Fraction(int(R[i, j])) for j in range(n)] for i in range(n)]
    x = [Fraction(int(t)) for t in v]
    if not upper_trans:
        for i in reversed(range(n)):
            x[i] = (x[i] - sum(Rf[i][j] * x[j] for j in range(i + 1, n))) / Rf[i][i]
    else:
        for i in range(n):
            x[i] = (x[i] - sum(Rf[j][i] * x[j] for j in range(i))) / Rf[i][i]
    return np.array([float(t) for t in x])


def test_trsv_exact_rationals():
    rng = np.random.default_rng(6)
    n = 9
    R = np.triu(rng.integers(-5, 6, (n, n))).astype(np.float64)
    R[np.diag_indices(n)] = rng.integers(1, 7, n) * rng.choice([-1, 1], n)
    v = rng.integers(-20, 21, n).astype(np.float64)
    np.testing.assert_allclose(oracle.trsv_upper(R, v), _frac_back_subst(R, v), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(oracle.trsv_upper_trans(R, v), _frac_back_subst(R, v, True), rtol=1e-14,
                               atol=1e-14)


def test_spmv_pair_matches_dense():
    rng = np.random.default_rng(7)
    A = random_sparse(500, 60, 7, rng)
    x = rng.standard_normal(60)
    u = rng.standard_normal(500)
    Ad = A.dense()
    np.testing.assert_allclose(oracle.spmv(A, x), Ad @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.spmv_trans(A, u), Ad.T @ u, rtol=1e-13, atol=1e-12)


# ----------------------------------------------------------------------------- LSQR

def test_lsqr_identity_preconditioner_matches_scipy_lsqr():
    """With M = I the oracle's recurrence is plain LSQR; SciPy implements the
    same Paige-Saunders recurrence, so early iterates agree to rounding and the
    converged solutions agree. (Mid-run Krylov iterates amplify rounding
    differences exponentially before convergence, so they are not compared.)"""
    rng = np.random.default_rng(8)
    A = random_sparse(300, 40, 6, rng, scale_exp=2.0)
    b = rng.standard_normal(300)
    sp = scipy.sparse.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    for k in (1, 2, 3, 5):
        x, info = oracle.lsqr(A, b, np.eye(A.n), "qr", fixed_iters=k)
        xs = scipy.sparse.linalg.lsqr(sp, b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        np.testing.assert_allclose(x, xs, rtol=1e-12, atol=1e-13 * np.abs(xs).max())
        assert info["iterations"] == k
    x, info = oracle.lsqr(A, b, np.eye(A.n), "qr", atol=1e-15, btol=1e-15, maxit=5000)
    xs = scipy.sparse.linalg.lsqr(sp, b, atol=1e-15, btol=1e-15, conlim=0, iter_lim=5000)[0]
    np.testing.assert_allclose(x, xs, rtol=1e-9, atol=1e-10 * np.abs(xs).max())


def _exact_ls(Ad, b):
    n = Ad.shape[1]
    M = [[Fraction(int(v)) for v in row] for row in Ad]
    bb = [Fraction(int(v)) for v in b]
    N = [[sum(M[k][i] * M[k][j] for k in range(len(M))) for j in range(n)] for i in range(n)]
    r = [sum(M[k][i] * bb[k] for k in range(len(M))) for i in range(n)]
    for c in range(n):                       # Gauss-Jordan in exact rationals
        piv = next(i for i in range(c, n) if N[i][c] != 0)
        N[c], N[piv] = N[piv], N[c]
        r[c], r[piv] = r[piv], r[c]
        for i in range(n):
            if i != c and N[i][c] != 0:
                f = N[i][c] / N[c][c]
                N[i] = [a - f * bq for a, bq in zip(N[i], N[c])]
                r[i] -= f * r[c]
    return np.array([float(r[i] / N[i][i]) for i in range(n)])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_csqrp_lsqr_tiny_exact(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 12, 4
    Ad = rng.integers(-6, 7, (m, n)).astype(np.float64)
    b = rng.integers(-10, 11, m).astype(np.float64)
    x_exact = _exact_ls(Ad, b)
    A = csr_from_dense(Ad)
    for variant in ("qr", "svd"):
        _, x, info = oracle.csqrp_lsqr(A, b, s=8, seed=seed + 3, variant=variant, tol=1e-15, maxit=50)
        np.testing.assert_allclose(x, x_exact, rtol=1e-13, atol=1e-13)


def test_lsqr_residual_monotone_cfg1():
    p = config_problem("cfg1")
    _, x, info, hist = oracle.csqrp_lsqr(p, p.b[0], seed=11, history=True)
    assert info["istop"] in (1, 2)
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    # the estimate ||r_k|| equals the true residual norm
    r = p.b[0] - oracle.spmv(p, x)
    assert abs(np.linalg.norm(r) - info["rnorm"]) < 1e-9 * np.linalg.norm(p.b[0])


def _cond(M):
    sv = np.linalg.svd(M, compute_uv=False)
    return sv[0] / sv[-1]


def test_theorem_3_3_iteration_bound():
    """Eq. 3.5: ||y_k - y_*||_{B^TB} <= 2 ((kappa-1)/(kappa+1))^k ||y_*||_{B^TB}
    with kappa = cond(B); k from that bound must reach tau in the A^TA norm."""
    rng = np.random.default_rng(9)
    A = random_sparse(3000, 80, 8, rng, scale_exp=8.0)
    b = rng.standard_normal(3000)
    Ad = A.dense()
    fac = oracle.factor(A, 320, seed=5)
    kappa = _cond(np.linalg.solve(fac["R"].T, Ad.T).T)
    tau = 1e-8
    q = (kappa - 1) / (kappa + 1)
    k = int(np.ceil((np.log(2) + abs(np.log(tau))) / abs(np.log(q))))
    x, info = oracle.lsqr(A, b, fac["R"], "qr", fixed_iters=k)
    x_star, _ = oracle.hhqr_solve(Ad, b)
    assert np.linalg.norm(Ad @ (x - x_star)) <= tau * np.linalg.norm(Ad @ x_star)


def test_theorem_3_2_condition_flat_under_column_scaling():
    rng = np.random.default_rng(10)
    base = random_sparse(2000, 50, 6, rng)
    conds = []
    for p in (0, 4, 8, 12):
        A = CSR(base.m, base.n, base.row_ptr, base.col,
                base.val * (10.0 ** (-p * np.arange(50) / 49))[base.col])
        fac = oracle.factor(A, 200, seed=3)
        B = np.linalg.solve(fac["R"].T, A.dense().T).T
        conds.append(_cond(B))
        if p >= 8:
            assert _cond(A.dense()) > 1e6
    assert max(conds) < 10 and max(conds) / min(conds) < 1.5


def test_bijective_sketch_gives_orthonormal_b():
    """With s = m the sketch is a signed permutation, so R is A's own R factor,
    A R^{-1} has orthonormal columns and LSQR converges in one iteration."""
    rng = np.random.default_rng(11)
    A = random_sparse(64, 10, 4, rng, scale_exp=6.0)
    b = rng.standard_normal(64)
    fac = oracle.factor(A, 64, seed=1)
    h, _ = oracle.hash_rows(64, 64, 1)
    if len(np.unique(h)) == 64:   # hash happens to be a bijection only sometimes
        B = np.linalg.solve(fac["R"].T, A.dense().T).T
        assert _cond(B) < 1 + 1e-8
    # make it bijective explicitly
    perm = rng.permutation(64).astype(np.int32)
    d = rng.choice([-1, 1], 64).astype(np.int8)
    R = oracle.r_factor(oracle.sketch(A, 64, perm, d))
    B = np.linalg.solve(R.T, A.dense().T).T
    assert _cond(B) < 1 + 1e-8
    x, info = oracle.lsqr(A, b, R, "qr", atol=1e-14, btol=1e-14, maxit=10)
    x_star = np.linalg.lstsq(A.dense(), b, rcond=None)[0]
    assert info["iterations"] <= 2
    np.testing.assert_allclose(x, x_star, rtol=1e-8, atol=1e-8 * np.abs(x_star).max())


def test_hhqr_matches_lstsq():
    rng = np.random.default_rng(12)
    Ad = rng.standard_normal((200, 30))
    b = rng.standard_normal(200)
    x, R = oracle.hhqr_solve(Ad, b)
    np.testing.assert_allclose(x, np.linalg.lstsq(Ad, b, rcond=None)[0], rtol=1e-12, atol=1e-13)


def test_cfg1_manufactured_solution_and_direct_agreement():
    p = config_problem("cfg1")
    _, x, info = oracle.csqrp_lsqr(p, p.b[0], seed=11)
    pts = np.random.default_rng(0).random((4000, 2))
    err = np.linalg.norm(p.evaluate(x, pts) - p.exact(pts)) / np.linalg.norm(p.exact(pts))
    assert err < 1e-3
    Ad = p.dense()
    x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
    assert np.linalg.norm(Ad @ (x - x_hh)) <= 1e-9 * np.linalg.norm(Ad @ x_hh)
    B = np.linalg.solve(oracle.factor(p, 1600, 11)["R"].T, Ad.T).T
    assert _cond(B) < 10


# ----------------------------------------------------------------------------- SVD variant

def test_jacobi_svd_matches_lapack():
    rng = np.random.default_rng(13)
    R = np.triu(rng.standard_normal((40, 40))) + 5 * np.eye(40)
    sigma, V, sweeps = oracle.jacobi_svd(R)
    np.testing.assert_allclose(sigma, np.linalg.svd(R, compute_uv=False), rtol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(40), atol=1e-12)
    U = R @ V / sigma
    np.testing.assert_allclose(U.T @ U, np.eye(40), atol=1e-11)


def test_cssvdp_rank_deficient_gives_min_norm_solution():
    """Theorem 3.1 / 3.4: with an exactly rank-deficient A the truncated SVD
    preconditioner recovers the rank and x = P (AP)^+ b is the minimum-norm LS solution."""
    rng = np.random.default_rng(14)
    base = rng.standard_normal((400, 20))
    Ad = np.concatenate([base, base[:, :3] @ rng.standard_normal((3, 4))], axis=1)   # rank 20 of 24
    Ad *= rng.random(Ad.shape) < 1.0
    b = rng.standard_normal(400)
    A = csr_from_dense(Ad)
    fac, x, info = oracle.csqrp_lsqr(A, b, s=96, seed=2, variant="svd", tol=1e-14, maxit=100)
    assert fac["r"] == 20
    x_mn = np.linalg.lstsq(Ad, b, rcond=None)[0]
    np.testing.assert_allclose(x, x_mn, rtol=1e-9, atol=1e-9 * np.abs(x_mn).max())
    assert _cond(Ad @ fac["F"]) < 10


def test_svd_and_qr_variants_agree_cfg1():
    p = config_problem("cfg1")
    _, xq, _ = oracle.csqrp_lsqr(p, p.b[0], seed=11)
    fac, xs, info = oracle.csqrp_lsqr(p, p.b[0], seed=11, variant="svd")
    Ad = p.dense()
    assert fac["r"] == p.n
    assert np.linalg.norm(Ad @ (xq - xs)) <= 1e-9 * np.linalg.norm(Ad @ xq)


# ----------------------------------------------------------------------------- adjoint

def test_adjoint_matches_finite_differences():
    prob = scaled_random_sparse(60, 8, per_row=4, cond_exp=2.0, seed=21)
    A = CSR(prob.m, prob.n, prob.row_ptr, prob.col, prob.val)
    b = prob.b[0]
    xt = prob.x_true

    def loss(vals, bb):
        Ad = CSR(A.m, A.n, A.row_ptr, A.col, vals).dense()
        x, _ = oracle.hhqr_solve(Ad, bb)
        return np.sum((x - xt) ** 2), x

    L0, x = loss(A.val, b)
    _, RA = oracle.hhqr_solve(A.dense(), b)
    lam, gb, gv = oracle.adjoint(A, b, x, RA, 2.0 * (x - xt))
    h = 1e-6
    fd_b = np.array([(loss(A.val, b + h * e)[0] - loss(A.val, b - h * e)[0]) / (2 * h) for e in np.eye(A.m)])
    np.testing.assert_allclose(gb, fd_b, rtol=1e-6, atol=1e-8 * np.abs(fd_b).max())
    fd_v = []
    for p in range(A.nnz):
        e = np.zeros(A.nnz)
        e[p] = h * abs(A.val[p])          # relative step: O(h^2) truncation
        fd_v.append((loss(A.val + e, b)[0] - loss(A.val - e, b)[0]) / (2 * e[p]))
    fd_v = np.array(fd_v)
    assert np.abs(gv - fd_v).max() <= 1e-5 * np.abs(fd_v).max()


# ----------------------------------------------------------------------------- warm start (Remark 3.1)

def test_lsqr_initial_guess_matches_scipy_lsqr():
    """LSQR from an initial point x0 (M = I) against SciPy's LSQR with the same x0: iterates and the
    converged solution (SciPy also keeps ||b|| of the original right-hand side in its stopping rule)."""
    rng = np.random.default_rng(3)
    A = random_sparse(300, 20, 5, rng)
    b = rng.standard_normal(300)
    x0 = rng.standard_normal(20)
    As = scipy.sparse.csr_matrix((A.val, A.col, A.row_ptr), shape=(A.m, A.n))
    for k in range(1, 6):
        x, _ = oracle.lsqr(A, b, np.eye(A.n), "qr", fixed_iters=k, x0=x0)
        xs = scipy.sparse.linalg.lsqr(As, b, x0=x0, atol=0, btol=0, iter_lim=k)[0]
        assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)
    x, info = oracle.lsqr(A, b, np.eye(A.n), "qr", atol=1e-14, btol=1e-14, maxit=500, x0=x0)
    ref = scipy.sparse.linalg.lsqr(As, b, x0=x0, atol=1e-14, btol=1e-14, iter_lim=500)
    assert np.linalg.norm(x - ref[0]) <= 1e-12 * np.linalg.norm(ref[0])
    assert info["iterations"] == ref[2]


def test_sketch_vector_is_the_sketch_of_b():
    """S b for a dense vector: a unit vector e_i lands as d(i) in bucket h(i); S is linear."""
    m, s = 50, 12
    h, d = oracle.hash_rows(m, s, 4)
    for i in (0, 7, 49):
        e = np.zeros(m)
        e[i] = 1.0
        want = np.zeros(s)
        want[h[i]] = d[i]
        assert np.array_equal(oracle.sketch_vector(e, s, h, d), want)
    rng = np.random.default_rng(1)
    b1, b2 = rng.integers(-5, 5, m).astype(float), rng.integers(-5, 5, m).astype(float)
    assert np.array_equal(oracle.sketch_vector(b1 + 2 * b2, s, h, d),
                          oracle.sketch_vector(b1, s, h, d) + 2 * oracle.sketch_vector(b2, s, h, d))


def test_sketch_solve_point_solves_the_sketched_problem():
    """x0 = R^-1 Q^T (S b) minimises ||S (A x - b)|| (its normal equations hold), and as a subspace
    embedding's sketch-and-solve point it fits the data nearly as well as the true solution."""
    rng = np.random.default_rng(8)
    A = random_sparse(4000, 60, 6, rng)
    Ad = A.dense()
    xt = rng.standard_normal(60)
    b = Ad @ xt + 0.1 * rng.standard_normal(4000)
    s = 240
    x0, Sb = oracle.sketch_solve(A, b, s, seed=2)
    h, d = oracle.hash_rows(A.m, s, 2)
    SA = oracle.sketch(A, s, h, d)
    g = SA.T @ (SA @ x0 - Sb)
    assert np.linalg.norm(g) <= 1e-10 * np.linalg.norm(SA) * np.linalg.norm(Sb)
    # the same point from the Householder R of the sketch: y0 = Q^T S b, x0 = R^-1 y0
    F, tau = oracle.householder_qr(np.column_stack([SA, Sb]))
    R = np.triu(F[:60, :60])
    y0 = F[:60, 60]
    assert np.linalg.norm(np.linalg.solve(R, y0) - x0) <= 1e-10 * np.linalg.norm(x0)
    x_star = np.linalg.lstsq(Ad, b, rcond=None)[0]
    assert np.linalg.norm(Ad @ x0 - b) <= 2.0 * np.linalg.norm(Ad @ x_star - b)


def test_warm_start_fewer_iterations_same_solution_cfg1():
    """Remark 3.1's starting point cuts LSQR iterations (the paper's elasticity and Poisson tables)
    and leaves the least-squares solution unchanged."""
    p = config_problem("cfg1")
    _, xc, ic = oracle.csqrp_lsqr(p, p.b[0], seed=11)
    fac, xw, iw = oracle.csqrp_lsqr(p, p.b[0], seed=11, warm=True)
    assert iw["iterations"] < ic["iterations"]
    Ad = p.dense()
    x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
    spread = np.linalg.norm(Ad @ (x_hh - xc)) / np.linalg.norm(Ad @ xc)
    assert np.linalg.norm(Ad @ (xw - xc)) <= max(1e-10, 2 * spread) * np.linalg.norm(Ad @ xc)
    assert abs(np.linalg.norm(p.b[0] - Ad @ xw) - np.linalg.norm(p.b[0] - Ad @ xc)) <= 1e-12 * np.linalg.norm(p.b[0])


# ----------------------------------------------------------------------------- explicit form (Algorithm 1 step 4)

def test_explicit_b_times_r_is_a_and_well_conditioned():
    """B = A R^-1 formed row by row satisfies B R = A, and cond(B) stays below 10 (Theorem 3.2)."""
    p = config_problem("cfg1")
    fac = oracle.factor(p, 4 * p.n, 11)
    B = oracle.form_b(p, fac)
    Ad = p.dense()
    assert np.linalg.norm(B @ fac["R"] - Ad) <= 1e-12 * np.linalg.norm(Ad)
    sv = np.linalg.svd(B, compute_uv=False)
    assert sv[0] / sv[-1] < 10


def test_explicit_form_solution_matches_direct_and_implicit():
    p = config_problem("cfg1")
    fac = oracle.factor(p, 4 * p.n, 11)
    x, y, info = oracle.explicit_lsqr(p, p.b[0], fac)
    Ad = p.dense()
    x_hh, _ = oracle.hhqr_solve(Ad, p.b[0])
    _, xi, _ = oracle.csqrp_lsqr(p, p.b[0], seed=11)
    spread = np.linalg.norm(Ad @ (x_hh - xi)) / np.linalg.norm(Ad @ xi)
    assert np.linalg.norm(Ad @ (x - x_hh)) <= max(1e-10, 2 * spread) * np.linalg.norm(Ad @ x_hh)
    assert info["istop"] in (1, 2)
    # M = I on a tiny exact problem: the explicit form with R = I is plain LSQR
    rng = np.random.default_rng(2)
    A = random_sparse(60, 5, 3, rng)
    b = rng.standard_normal(60)
    x1, _, _ = oracle.explicit_lsqr(A, b, dict(kind="qr", R=np.eye(5), F=np.eye(5)), tol=1e-15, maxit=50)
    np.testing.assert_allclose(x1, np.linalg.lstsq(A.dense(), b, rcond=None)[0], rtol=1e-10, atol=1e-12)


def test_threaded_qr_is_bit_identical():
    """The oracle's one OpenMP loop (trailing columns of the Householder QR) leaves every column's
    arithmetic in the serial order, so any thread count gives the same bits."""
    M = np.random.default_rng(3).standard_normal((700, 300))
    prev = oracle.set_threads(0)
    oracle.set_threads(1)
    F1, t1 = oracle.householder_qr(M)
    oracle.set_threads(4)
    F4, t4 = oracle.householder_qr(M)
    oracle.set_threads(prev)
    assert np.array_equal(F1, F4) and np.array_equal(t1, t4)


def test_restart_reaches_the_dense_solution():
    """The implicit form's rounding floor moves with the sketch: on a 3x2-box RFM system (cond ~1e9)
    the first solves of two sketches end ~1e-10 apart in the A-norm and as far from the dense
    Householder solution; one LSQR restart from the solution found (the correction from
    r = b - A x) brings both to the dense solution (the same point by an independent route)."""
    p = poisson2d(3, 2, 150, 24, 24, R=2.0, seed=2)
    Ad = p.dense()
    b = p.b[0]
    an = lambda x, r: np.linalg.norm(Ad @ (x - r)) / np.linalg.norm(Ad @ r)
    first, restarted = [], []
    for seed in (1, 2):
        first.append(oracle.csqrp_lsqr(p, b, seed=seed)[1])
        fac, x, info = oracle.csqrp_lsqr(p, b, seed=seed, refine=1)
        assert info["iterations_refine"] > 0
        restarted.append(x)
    x_hh, _ = oracle.hhqr_solve(Ad, b)
    assert an(first[0], first[1]) > 1e-11
    assert an(restarted[0], restarted[1]) <= 1e-13
    for x in restarted:
        assert an(x, x_hh) <= 1e-13
