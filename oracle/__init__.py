"""CPU oracle for the count-sketch preconditioned LSQR method.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may import this package; the product path never does. The arithmetic
lives in ``csls_oracle.c`` (plain scalar C, binary64, no fused multiply-add),
loaded here with ctypes; this module only marshals arrays and chains the steps
of Algorithm 1 (CSQRP-LSQR) and Algorithm 2 (CSSVDP-LSQR) in the paper's order.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csls_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libcsls_oracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with gcc (-O2 -ffp-contract=off -fopenmp); returns the .so path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u64, i64, i32, dbl, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
        sig = {
            "orc_set_threads": (ctypes.c_int, [ctypes.c_int]),
            "orc_splitmix64_mix": (u64, [u64]),
            "orc_splitmix64_output": (u64, [u64, u64]),
            "orc_hash": (None, [i64, i64, u64, vp, vp]),
            "orc_sketch": (None, [i64, i64, vp, vp, vp, i64, vp, vp, vp, i64]),
            "orc_sketch_f32": (None, [i64, i64, vp, vp, vp, i64, vp, vp, vp, i64]),
            "orc_householder_qr": (None, [i64, i64, vp, i64, vp]),
            "orc_householder_qr_f32": (None, [i64, i64, vp, i64, vp]),
            "orc_extract_r": (None, [i64, vp, i64, vp, i64]),
            "orc_trsv_upper": (None, [i64, vp, i64, vp]),
            "orc_trsv_upper_trans": (None, [i64, vp, i64, vp]),
            "orc_spmv": (None, [i64, vp, vp, vp, vp, vp]),
            "orc_spmv_trans": (None, [i64, i64, vp, vp, vp, vp, vp]),
            "orc_lsqr": (None, [i64, i64, vp, vp, vp, vp, ctypes.c_int, vp, i64, i64, dbl, dbl, i64, i64,
                                vp, vp, vp, vp]),
            "orc_hhqr_solve": (None, [i64, i64, vp, i64, vp, vp, vp]),
            "orc_jacobi_svd": (ctypes.c_int, [i64, vp, i64, vp, vp, i64, ctypes.c_int]),
            "orc_svd_precond": (i64, [i64, vp, vp, i64, dbl, vp, i64]),
            "orc_adjoint": (None, [i64, i64, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _csr(A):
    return (np.ascontiguousarray(A.row_ptr, dtype=np.int64), np.ascontiguousarray(A.col, dtype=np.int32),
            np.ascontiguousarray(A.val, dtype=np.float64))


# --------------------------------------------------------------------------- primitives

def set_threads(nthreads):
    """Threads of the Householder QR's column loop (results do not depend on it); returns the count."""
    return int(_load().orc_set_threads(int(nthreads)))


def splitmix64_output(seed, i):
    return int(_load().orc_splitmix64_output(seed, i))


def hash_rows(m, s, seed):
    """Bucket h(i) in [0, s) and sign d(i) in {-1, +1} for rows i < m (Definition 2.3)."""
    h = np.empty(m, dtype=np.int32)
    d = np.empty(m, dtype=np.int8)
    _load().orc_hash(m, s, seed, _p(h), _p(d))
    return h, d


def sketch(A, s, h, d, dtype=np.float64):
    """SA (s x n, column-major) with rows visited in ascending order (Algorithm 1 step 2)."""
    rp, cl, vl = _csr(A)
    h = np.ascontiguousarray(h, dtype=np.int32)
    d = np.ascontiguousarray(d, dtype=np.int8)
    out = np.empty((s, A.n), dtype=dtype, order="F")
    fn = _load().orc_sketch if dtype == np.float64 else _load().orc_sketch_f32
    fn(A.m, A.n, _p(rp), _p(cl), _p(vl), s, _p(h), _p(d), _p(out), s)
    return out


def householder_qr(M):
    """Unblocked Householder QR of a column-major copy; returns (factored, tau)."""
    dtype = M.dtype
    F = np.array(M, dtype=dtype, order="F", copy=True)
    s, n = F.shape
    tau = np.empty(min(s, n), dtype=dtype)
    fn = _load().orc_householder_qr if dtype == np.float64 else _load().orc_householder_qr_f32
    fn(s, n, _p(F), s, _p(tau))
    return F, tau


def r_factor(M):
    """Sign-normalised (non-negative diagonal) R of M, in binary64."""
    F, _ = householder_qr(M)
    n = F.shape[1]
    F64 = np.asfortranarray(F, dtype=np.float64)   # no second copy of a binary64 factor
    R = np.empty((n, n), dtype=np.float64, order="F")
    _load().orc_extract_r(n, _p(F64), F64.shape[0], _p(R), n)
    return R


def trsv_upper(R, v):
    R = np.asfortranarray(R, dtype=np.float64)
    x = np.array(v, dtype=np.float64, copy=True)
    _load().orc_trsv_upper(R.shape[0], _p(R), R.shape[0], _p(x))
    return x


def trsv_upper_trans(R, v):
    R = np.asfortranarray(R, dtype=np.float64)
    x = np.array(v, dtype=np.float64, copy=True)
    _load().orc_trsv_upper_trans(R.shape[0], _p(R), R.shape[0], _p(x))
    return x


def spmv(A, x):
    rp, cl, vl = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.m)
    _load().orc_spmv(A.m, _p(rp), _p(cl), _p(vl), _p(x), _p(y))
    return y


def spmv_trans(A, u):
    rp, cl, vl = _csr(A)
    u = np.ascontiguousarray(u, dtype=np.float64)
    y = np.empty(A.n)
    _load().orc_spmv_trans(A.m, A.n, _p(rp), _p(cl), _p(vl), _p(u), _p(y))
    return y


def lsqr(A, b, F, kind="qr", atol=1e-12, btol=1e-12, maxit=None, fixed_iters=0, history=False, x0=None):
    """Implicit-form preconditioned LSQR: B = A R^{-1} (kind 'qr', F = R) or
    B = A P (kind 'svd', F = P, n x r), from x0 (default 0). Returns (x, info[, rnorm history])."""
    rp, cl, vl = _csr(A)
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    F = np.asfortranarray(F, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    maxit = A.n if maxit is None else maxit
    x = np.empty(A.n)
    out = np.empty(6)
    nhist = (fixed_iters if fixed_iters > 0 else maxit) + 1
    hist = np.zeros(nhist)
    r = F.shape[1]
    _load().orc_lsqr(A.m, A.n, _p(rp), _p(cl), _p(vl), _p(b), 0 if kind == "qr" else 1, _p(F), F.shape[0], r,
                     atol, btol, maxit, fixed_iters, _p(x0) if x0 is not None else None, _p(x), _p(out),
                     _p(hist))
    info = dict(iterations=int(out[0]), istop=int(out[1]), rnorm=out[2], arnorm=out[3], anorm=out[4],
                ynorm=out[5])
    if history:
        return x, info, hist[: info["iterations"] + 1]
    return x, info


def hhqr_solve(Ad, b):
    """Dense Householder least-squares solve; returns (x, sign-normalised R of A)."""
    Ad = np.asfortranarray(Ad, dtype=np.float64)
    m, n = Ad.shape
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n)
    R = np.empty((n, n), order="F")
    _load().orc_hhqr_solve(m, n, _p(Ad), m, _p(b), _p(x), _p(R))
    return x, R


def jacobi_svd(R, max_sweeps=60):
    R = np.asfortranarray(R, dtype=np.float64)
    n = R.shape[0]
    sigma = np.empty(n)
    V = np.empty((n, n), order="F")
    sweeps = _load().orc_jacobi_svd(n, _p(R), n, _p(sigma), _p(V), n, max_sweeps)
    return sigma, V, sweeps


def svd_precond(sigma, V, rcond):
    n = V.shape[0]
    V = np.asfortranarray(V, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    P = np.zeros((n, n), order="F")
    r = _load().orc_svd_precond(n, _p(sigma), _p(V), n, rcond, _p(P), n)
    return np.asfortranarray(P[:, :r]), int(r)


def adjoint(A, b, x, RA, g):
    """(lambda, dL/db, dL/dvals) for a loss with gradient g at the LS solution x."""
    rp, cl, vl = _csr(A)
    RA = np.asfortranarray(RA, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    lam = np.empty(A.n)
    gb = np.empty(A.m)
    gv = np.empty(A.nnz)
    _load().orc_adjoint(A.m, A.n, _p(rp), _p(cl), _p(vl), _p(b), _p(x), _p(RA), RA.shape[0], _p(g),
                        _p(lam), _p(gb), _p(gv))
    return lam, gb, gv


# --------------------------------------------------------------------------- the method

def default_rcond(s, n):
    """RCOND = max(s, n) * unit roundoff (LAPACK least-squares convention)."""
    return max(s, n) * np.finfo(np.float64).eps / 2


def sketch_size(A, gamma=4.0, s=None):
    """s = gamma n (Algorithm 1 step 1), clamped to m when gamma n would exceed it."""
    if s is None:
        s = int(round(gamma * A.n))
    return int(min(s, A.m))


def factor(A, s, seed, variant="qr", prec="f64", rcond=None):
    """Algorithm 1 steps 1-3 (variant 'qr') or Algorithm 2 steps 1-3 (variant 'svd')."""
    h, d = hash_rows(A.m, s, seed)
    SA = sketch(A, s, h, d, np.float64 if prec == "f64" else np.float32)
    R = r_factor(SA)
    if variant == "qr":
        return dict(kind="qr", F=R, R=R, s=s, SA=SA)
    sigma, V, _ = jacobi_svd(R)
    rc = default_rcond(s, A.n) if rcond is None else rcond
    P, r = svd_precond(sigma, V, rc)
    return dict(kind="svd", F=P, R=R, sigma=sigma, V=V, r=r, s=s, SA=SA)


def sketch_solve(A, b, s, seed, fac=None):
    """x0 = argmin ||S (A x - b)||: the sketch-and-solve point that Remark 3.1's y0 = Q^T (S b)
    stands for (y0 = R x0), from LAPACK's least squares on the sketched system."""
    h, d = hash_rows(A.m, s, seed)
    SA = fac["SA"] if fac is not None else sketch(A, s, h, d)
    Sb = sketch_vector(b, s, h, d)
    return np.linalg.lstsq(SA, Sb, rcond=None)[0], Sb


def sketch_vector(b, s, h, d):
    """S b for a dense m-vector (Definition 2.3; rows summed in ascending order per bucket)."""
    m = len(b)
    one = _Csr1(m, np.arange(m + 1, dtype=np.int64), np.zeros(m, np.int32), np.ascontiguousarray(b, np.float64))
    return sketch(one, s, h, d)[:, 0]


class _Csr1:
    """b as an m x 1 CSR matrix (one nonzero per row)."""

    def __init__(self, m, row_ptr, col, val):
        self.m, self.n, self.row_ptr, self.col, self.val = m, 1, row_ptr, col, val

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def form_b(A, fac):
    """The explicit preconditioned matrix of Algorithm 1 step 4 / Algorithm 2 step 4: B = A R^-1 (each
    row b_i solves R^T b_i = a_i by substitution) or B = A P. Dense m x r, column-major."""
    Ad = np.zeros((A.m, A.n))
    rows = np.repeat(np.arange(A.m), np.diff(A.row_ptr))
    Ad[rows, A.col] = A.val
    if fac["kind"] == "svd":
        return np.asfortranarray(Ad @ fac["F"])
    R = fac["R"]
    B = np.empty((A.m, A.n), order="F")
    for i in range(A.m):
        B[i, :] = trsv_upper_trans(R, Ad[i, :])
    return B


class _Dense:
    """A dense matrix as CSR with every entry stored (for the oracle's LSQR on B)."""

    def __init__(self, B):
        m, n = B.shape
        self.m, self.n = m, n
        self.row_ptr = np.arange(m + 1, dtype=np.int64) * n
        self.col = np.tile(np.arange(n, dtype=np.int32), m)
        self.val = np.ascontiguousarray(B).reshape(-1)

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def explicit_lsqr(A, b, fac, tol=1e-12, maxit=None, fixed_iters=0):
    """LSQR on the formed B (Algorithm 1 step 5), then x = R^-1 y or P y (step 6). Returns (x, y, info)."""
    B = form_b(A, fac)
    r = B.shape[1]
    y, info = lsqr(_Dense(B), b, np.eye(r), "qr", atol=tol, btol=tol,
                   maxit=(A.n if maxit is None else maxit), fixed_iters=fixed_iters)
    x = fac["F"] @ y if fac["kind"] == "svd" else trsv_upper(fac["R"], y)
    return x, y, info


def csqrp_lsqr(A, b, gamma=4.0, s=None, seed=1, variant="qr", prec="f64", tol=1e-12, maxit=None,
               fixed_iters=0, history=False, warm=False, refine=0):
    """Full CSQRP-LSQR (Algorithm 1) / CSSVDP-LSQR (Algorithm 2) in the implicit form; with warm=True
    LSQR starts from the sketch-and-solve point of Remark 3.1. refine > 0 restarts LSQR that many times
    from the solution found (the same initial-point form, x0 = the previous x): each restart solves for
    the correction from r = b - A x. info["iterations_refine"] counts the restarts' iterations."""
    s = sketch_size(A, gamma, s)
    fac = factor(A, s, seed, variant, prec)
    x0 = None
    if warm:
        x0, _ = sketch_solve(A, b, s, seed, fac)
        fac = dict(fac, x0=x0)
    res = lsqr(A, b, fac["F"], fac["kind"], atol=tol, btol=tol, maxit=maxit, fixed_iters=fixed_iters,
               history=history, x0=x0)
    if refine > 0:
        x, info = res[0], dict(res[1])
        its = 0
        for _ in range(refine):
            x, inf2 = lsqr(A, b, fac["F"], fac["kind"], atol=tol, btol=tol, maxit=maxit, x0=x)
            its += inf2["iterations"]
        info.update(iterations_refine=its, rnorm=inf2["rnorm"], istop=inf2["istop"])
        res = (x, info) + tuple(res[2:])
    return (fac,) + tuple(res)
