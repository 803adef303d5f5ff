"""Thin ctypes binding of the csls C ABI (include/csls.h).

Functions named ``csls_*`` mirror the C entry points one to one; they only
marshal torch CUDA tensors into pointers and sizes. Every step of the method
runs in the CUDA library: there is no Python or CPU fallback, and loading fails
loudly when the compiled library is missing.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcsls.so")

CSLS_OK = 0
STATUS_NAMES = {
    0: "CSLS_OK", 1: "CSLS_ERR_ARG", 2: "CSLS_ERR_RANK_DEFICIENT", 3: "CSLS_ERR_NOT_CONVERGED",
    4: "CSLS_ERR_BREAKDOWN", 5: "CSLS_ERR_NONFINITE", 6: "CSLS_ERR_PRECOND_GUARD", 7: "CSLS_ERR_TIMEOUT",
    8: "CSLS_ERR_CUDA", 9: "CSLS_ERR_WORKSPACE",
}
VARIANT = {"qr": 0, "svd": 1}
PREC = {"f64": 0, "f32": 1, "f64emu": 2}


class CslsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "%s failed: %s" % (where, _lib().csls_status_string(status).decode())
        if status == 8:   # CSLS_ERR_CUDA: the runtime's own message
            msg += " [%s]" % _lib().csls_last_cuda_error().decode()
        super().__init__(msg)


class csls_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class csls_opts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("s", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("variant", ctypes.c_int), ("factor_prec", ctypes.c_int), ("rcond", ctypes.c_double),
                ("atol", ctypes.c_double), ("btol", ctypes.c_double), ("maxit", ctypes.c_int64),
                ("fixed_iters", ctypes.c_int64), ("guard_cond", ctypes.c_double), ("spin_limit", ctypes.c_int64),
                ("check_every", ctypes.c_int64), ("time_kernels", ctypes.c_int64), ("warm_start", ctypes.c_int64),
                ("refine", ctypes.c_int64)]


class csls_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("istop", ctypes.c_int), ("iterations", ctypes.c_int64),
                ("s", ctypes.c_int64), ("r", ctypes.c_int64), ("bnorm", ctypes.c_double),
                ("rnorm", ctypes.c_double), ("arnorm", ctypes.c_double), ("anorm", ctypes.c_double),
                ("ynorm", ctypes.c_double), ("cond_est", ctypes.c_double), ("rdiag_min", ctypes.c_double),
                ("rdiag_max", ctypes.c_double), ("ms_sketch", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("launches", ctypes.c_int64),
                ("kern_ms", ctypes.c_double * 3), ("kern_launches", ctypes.c_int64 * 3),
                ("kern_flop", ctypes.c_double * 3), ("iterations_refine", ctypes.c_int64)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, ctypes.Array) else v
        return out


EXPORTS = {
    "csls_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "csls_last_cuda_error": (ctypes.c_char_p, []),
    "csls_opts_default": (None, [ctypes.c_void_p]),
    "csls_sketch_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "csls_sketch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "csls_sketch_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "csls_factor_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "csls_factor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "csls_factor_warm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "csls_factor_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "csls_rfm_assemble_workspace": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p]),
    "csls_rfm_nnz": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "csls_rfm_assemble": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "csls_form_b_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "csls_form_b": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "csls_solve_explicit_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "csls_solve_explicit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "csls_factor_view": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 7),
    "csls_precond_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "csls_spmv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "csls_apply_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "csls_read_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "csls_solve_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "csls_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "csls_backward_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "csls_batch_solve_workspace": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "csls_batch_solve": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "csls_autotune_spmv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "csls_factor_set_spmv_groups": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "csls_solve_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
}

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcsls.so is not built (%s); run paper_2409_15818_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(status, where):
    if status != CSLS_OK:
        raise CslsError(status, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes, device):
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------------- matrix and options

class Csr:
    """A device CSR matrix in the layout the library expects (int64 row_ptr,
    int32 columns ascending per row, float64 values)."""

    def __init__(self, row_ptr, col, val, m, n):
        self.row_ptr = row_ptr.to(torch.int64).contiguous()
        self.col = col.to(torch.int32).contiguous()
        self.val = val.to(torch.float64).contiguous()
        self.m, self.n = int(m), int(n)
        assert self.row_ptr.is_cuda and self.col.is_cuda and self.val.is_cuda, "csls needs CUDA tensors"

    @classmethod
    def from_numpy(cls, row_ptr, col, val, m, n, device="cuda"):
        return cls(torch.as_tensor(row_ptr, device=device), torch.as_tensor(col, device=device),
                   torch.as_tensor(val, device=device), m, n)

    @classmethod
    def from_torch_sparse(cls, a):
        a = a.to_sparse_csr() if a.layout != torch.sparse_csr else a
        return cls(a.crow_indices(), a.col_indices(), a.values(), a.shape[0], a.shape[1])

    @property
    def nnz(self):
        return int(self.col.numel())

    def with_values(self, val):
        return Csr(self.row_ptr, self.col, val, self.m, self.n)

    def struct(self):
        return csls_csr(self.m, self.n, self.nnz, self.row_ptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr())


def make_opts(gamma=4.0, s=0, seed=1, variant="qr", prec="f64", rcond=0.0, atol=1e-12, btol=1e-12, maxit=0,
              fixed_iters=0, guard_cond=10.0, spin_limit=20_000_000, check_every=16, time_kernels=0, warm_start=0,
              refine=0, tol=None):
    o = csls_opts()
    _lib().csls_opts_default(ctypes.byref(o))
    if tol is not None:
        atol = btol = tol
    o.gamma, o.s, o.seed = float(gamma), int(s), int(seed)
    o.variant, o.factor_prec = VARIANT[variant], PREC[prec]
    o.rcond, o.atol, o.btol = float(rcond), float(atol), float(btol)
    o.maxit, o.fixed_iters = int(maxit), int(fixed_iters)
    o.guard_cond, o.spin_limit, o.check_every = float(guard_cond), int(spin_limit), int(check_every)
    o.time_kernels = int(time_kernels)
    o.warm_start = int(warm_start)
    o.refine = int(refine)
    return o


# --------------------------------------------------------------------------- C ABI mirrors

def csls_status_string(status):
    return _lib().csls_status_string(int(status)).decode()


def csls_sketch(A, s, seed, prec="f64", SA=None, ld=None, stream=None):
    """SA = S A (s x n column-major); returns the tensor viewed as (n, ld) row-major storage."""
    ld = int(ld or s)
    dtype = torch.float32 if prec == "f32" else torch.float64
    if SA is None:
        SA = torch.empty((A.n, ld), dtype=dtype, device=A.val.device)
    a = A.struct()
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_sketch_workspace(ctypes.byref(a), s, ctypes.byref(nbytes)), "csls_sketch_workspace")
    work = _workspace(nbytes.value, A.val.device)
    _check(_lib().csls_sketch(ctypes.byref(a), s, seed, PREC[prec], _ptr(SA), ld, _ptr(work), work.numel(),
                              _stream(stream)), "csls_sketch")
    return SA


def csls_sketch_noalloc(A, s, seed, prec="f64", SA=None, ld=None, stream=None, raise_on_error=True):
    """csls_sketch on the library's fixed scratch area (no workspace allocation);
    returns (SA, status)."""
    ld = int(ld or s)
    dtype = torch.float64 if prec == "f64" else torch.float32
    if SA is None:
        SA = torch.empty((A.n, ld), dtype=dtype, device=A.val.device)
    a = A.struct()
    st = _lib().csls_sketch_noalloc(ctypes.byref(a), s, seed, PREC[prec], _ptr(SA), ld, _stream(stream))
    if raise_on_error:
        _check(st, "csls_sketch_noalloc")
    return SA, st


class Factor:
    """Owns the persistent workspace and the library handle of csls_factor."""

    def __init__(self, handle, persist, A, opts, report):
        self.handle = handle
        self.persist = persist
        self.A = A
        self.opts = opts
        self.report = report

    def view(self):
        n, s, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        var, prec = ctypes.c_int(), ctypes.c_int()
        R, P = ctypes.c_void_p(), ctypes.c_void_p()
        _check(_lib().csls_factor_view(self.handle, ctypes.byref(n), ctypes.byref(s), ctypes.byref(r),
                                       ctypes.byref(var), ctypes.byref(prec), ctypes.byref(R), ctypes.byref(P)),
               "csls_factor_view")
        return dict(n=n.value, s=s.value, r=r.value, variant=var.value, prec=prec.value, R=R.value, P=P.value)

    def R(self):
        """Copy of R (n x n, upper triangular) as a torch tensor."""
        v = self.view()
        n = v["n"]
        dtype = torch.float64 if v["prec"] == 0 else torch.float32
        esz = 8 if v["prec"] == 0 else 4
        off = v["R"] - self.persist.data_ptr()
        raw = self.persist[off: off + n * n * esz].view(dtype).view(n, n)   # column-major R = row-major R^T
        return raw.t().clone()

    def P(self):
        v = self.view()
        if not v["P"]:
            return None
        n, r = v["n"], v["r"]
        off = v["P"] - self.persist.data_ptr()
        raw = self.persist[off: off + n * r * 8].view(torch.float64).view(r, n)
        return raw.t().clone()

    def __del__(self):
        try:
            if self.handle:
                _lib().csls_factor_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def csls_factor(A, opts=None, stream=None, **kw):
    opts = opts or make_opts(**kw)
    a = A.struct()
    pb, tb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib().csls_factor_workspace(ctypes.byref(a), ctypes.byref(opts), ctypes.byref(pb), ctypes.byref(tb)),
           "csls_factor_workspace")
    dev = A.val.device
    persist = _workspace(pb.value, dev)
    temp = _workspace(tb.value, dev)
    handle = ctypes.c_void_p()
    rep = csls_report()
    st = _lib().csls_factor(ctypes.byref(a), ctypes.byref(opts), _ptr(persist), persist.numel(),
                                            _ptr(temp), temp.numel(), ctypes.byref(handle), ctypes.byref(rep),
                                            _stream(stream))
    del temp
    _check(st, "csls_factor")
    return Factor(handle, persist, A, opts, rep.as_dict())


def csls_factor_warm(A, b, opts=None, stream=None, **kw):
    """csls_factor plus Remark 3.1's starting point: returns (factor, x0) with
    x0 = argmin ||S (A x - b)|| from the QR of the augmented sketch [SA, Sb]."""
    opts = opts or make_opts(**kw)
    a = A.struct()
    pb, tb = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib().csls_factor_workspace(ctypes.byref(a), ctypes.byref(opts), ctypes.byref(pb), ctypes.byref(tb)),
           "csls_factor_workspace")
    dev = A.val.device
    persist = _workspace(pb.value, dev)
    temp = _workspace(tb.value, dev)
    b = b.contiguous()
    x0 = torch.empty(A.n, dtype=torch.float64, device=dev)
    handle = ctypes.c_void_p()
    rep = csls_report()
    st = _lib().csls_factor_warm(ctypes.byref(a), _ptr(b), ctypes.byref(opts), _ptr(persist), persist.numel(),
                                 _ptr(temp), temp.numel(), ctypes.byref(handle), _ptr(x0), ctypes.byref(rep),
                                 _stream(stream))
    del temp
    _check(st, "csls_factor_warm")
    return Factor(handle, persist, A, opts, rep.as_dict()), x0


def csls_rfm_assemble(dim, r_half, J, k, c, rows, stream=None):
    """CSR of an RFM system assembled on the device. k (boxes, J, dim) and c (boxes, J) are
    float64 tensors on the device; rows is a uint8 device tensor holding the csls_rfm_row
    descriptors (40 bytes each). Returns a Csr."""
    nrows = rows.numel() // 40
    assert rows.numel() == 40 * nrows and rows.dtype == torch.uint8
    dev = k.device
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_rfm_assemble_workspace(nrows, ctypes.byref(nbytes)), "csls_rfm_assemble_workspace")
    work = _workspace(nbytes.value, dev)
    nnz_h = ctypes.c_int64()
    _check(_lib().csls_rfm_nnz(nrows, _ptr(rows), int(J), _ptr(work), work.numel(), ctypes.byref(nnz_h),
                               _stream(stream)), "csls_rfm_nnz")
    nnz = nnz_h.value
    row_ptr = torch.empty(nrows + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz, 1), dtype=torch.float64, device=dev)
    rh = (ctypes.c_double * dim)(*[float(v) for v in r_half])
    _check(_lib().csls_rfm_assemble(int(dim), rh, int(J), _ptr(k.contiguous()), _ptr(c.contiguous()), nrows,
                                    _ptr(rows), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(work), work.numel(),
                                    _stream(stream)), "csls_rfm_assemble")
    n = int(k.shape[0]) * int(J)
    return Csr(row_ptr, col[:nnz], val[:nnz], nrows, n)


def csls_form_b(F, A, stream=None):
    """B = A R^-1 (or A P) as a dense tensor; returns the (r, m) row-major view of the column-major B."""
    v = F.view()
    r = v["r"]
    B = torch.empty((r, A.m), dtype=torch.float64, device=A.val.device)
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_form_b_workspace(F.handle, ctypes.byref(nbytes)), "csls_form_b_workspace")
    work = _workspace(nbytes.value, A.val.device)
    a = A.struct()
    _check(_lib().csls_form_b(F.handle, ctypes.byref(a), _ptr(B), A.m, _ptr(work), work.numel(), _stream(stream)),
           "csls_form_b")
    return B


def csls_solve_explicit(F, B, b, opts=None, stream=None, raise_on_error=True, **kw):
    """LSQR on the formed B (from csls_form_b), x = R^-1 y or P y; returns (x, report dict)."""
    opts = opts or make_opts(**kw)
    m = B.shape[1]
    x = torch.empty(F.view()["n"], dtype=torch.float64, device=b.device)
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_solve_explicit_workspace(F.handle, ctypes.byref(nbytes)), "csls_solve_explicit_workspace")
    work = _workspace(nbytes.value, b.device)
    rep = csls_report()
    st = _lib().csls_solve_explicit(F.handle, _ptr(B), m, _ptr(b.contiguous()), _ptr(x), ctypes.byref(opts),
                                    _ptr(work), work.numel(), ctypes.byref(rep), _stream(stream))
    if raise_on_error:
        _check(st, "csls_solve_explicit")
    out = rep.as_dict()
    out["status"] = st
    return x, out


def csls_precond_apply(F, v, trans=False, stream=None):
    z = torch.empty_like(v)
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_apply_workspace(F.handle, ctypes.byref(nbytes)), "csls_apply_workspace")
    work = _workspace(nbytes.value, v.device)
    _check(_lib().csls_precond_apply(F.handle, int(bool(trans)), _ptr(v), _ptr(z), _ptr(work), work.numel(),
                                     _stream(stream)), "csls_precond_apply")
    return z


def csls_spmv(F, A, x, trans=False, stream=None, y=None):
    if y is None:
        y = torch.empty(A.n if trans else A.m, dtype=torch.float64, device=x.device)
    a = A.struct()
    _check(_lib().csls_spmv(F.handle, ctypes.byref(a), int(bool(trans)), _ptr(x), _ptr(y), _stream(stream)),
           "csls_spmv")
    return y


def csls_read_probe(buf, ctas_per_sm=2, unroll=8, stream=None, partials=None):
    """Streaming read of a device buffer (a multiple of 8 bytes, 16-byte aligned) by the library's
    probe kernel; returns the per-CTA 64-bit wrap-around sums (int64 tensor, reinterpreted)."""
    count = buf.numel() * buf.element_size() // 8
    if partials is None:
        sms = torch.cuda.get_device_properties(buf.device).multi_processor_count
        partials = torch.empty(sms * ctas_per_sm, dtype=torch.int64, device=buf.device)
    _check(_lib().csls_read_probe(_ptr(buf), count, int(ctas_per_sm), int(unroll), _ptr(partials), _stream(stream)),
           "csls_read_probe")
    return partials


def csls_solve(F, A, b, opts=None, x=None, stream=None, raise_on_error=True, **kw):
    """x (n,) or (nrhs, n) for b (m,) or (nrhs, m); returns (x, report dict)."""
    opts = opts or make_opts(**kw)
    b2 = b.reshape(-1, A.m).contiguous()
    nrhs = b2.shape[0]
    if x is None:
        x = torch.empty((nrhs, A.n), dtype=torch.float64, device=b.device)
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_solve_workspace(F.handle, nrhs, ctypes.byref(nbytes)), "csls_solve_workspace")
    work = _workspace(nbytes.value, b.device)
    rep = csls_report()
    a = A.struct()
    st = _lib().csls_solve(F.handle, ctypes.byref(a), _ptr(b2), nrhs, A.m, _ptr(x), A.n, ctypes.byref(opts),
                           _ptr(work), work.numel(), ctypes.byref(rep), _stream(stream))
    if raise_on_error:
        _check(st, "csls_solve")
    out = rep.as_dict()
    out["status"] = st
    return (x.reshape(b.shape[:-1] + (A.n,)) if b.dim() == 1 else x), out


def csls_solve_backward(F, A, b, x, grad_x, want_b=True, want_val=True, opts=None, stream=None, **kw):
    opts = opts or make_opts(**kw)
    gb = torch.empty(A.m, dtype=torch.float64, device=b.device) if want_b else None
    gv = torch.empty(A.nnz, dtype=torch.float64, device=b.device) if want_val else None
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_backward_workspace(F.handle, ctypes.byref(nbytes)), "csls_backward_workspace")
    work = _workspace(nbytes.value, b.device)
    rep = csls_report()
    a = A.struct()
    _check(_lib().csls_solve_backward(F.handle, ctypes.byref(a), _ptr(b.contiguous()), _ptr(x.contiguous()),
                                      _ptr(grad_x.contiguous()), _ptr(gb), _ptr(gv), ctypes.byref(opts),
                                      _ptr(work), work.numel(), ctypes.byref(rep), _stream(stream)),
           "csls_solve_backward")
    return gb, gv, rep.as_dict()


# --------------------------------------------------------------------------- batches and autotuning

def csls_batch_solve(factors, As, bs, opts=None, stream=None, raise_on_error=True, **kw):
    """Solve many independent problems (each with its own factor) in one CUDA-graph
    launch; returns (list of x, list of report dicts)."""
    opts = opts or make_opts(**kw)
    count = len(factors)
    handles = (ctypes.c_void_p * count)(*[f.handle.value for f in factors])
    csrs = (csls_csr * count)(*[A.struct() for A in As])
    bs = [b.contiguous() for b in bs]
    xs = [torch.empty(A.n, dtype=torch.float64, device=b.device) for A, b in zip(As, bs)]
    bp = (ctypes.c_void_p * count)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * count)(*[x.data_ptr() for x in xs])
    nbytes = ctypes.c_size_t()
    _check(_lib().csls_batch_solve_workspace(count, handles, ctypes.byref(nbytes)), "csls_batch_solve_workspace")
    work = _workspace(nbytes.value, bs[0].device)
    reps = (csls_report * count)()
    st = _lib().csls_batch_solve(count, handles, csrs, bp, xp, ctypes.byref(opts), _ptr(work), work.numel(), reps,
                                 _stream(stream))
    if raise_on_error:
        _check(st, "csls_batch_solve")
    return xs, [r.as_dict() for r in reps], st


def _tune_key(A):
    return "%dx%d:%d:%s" % (A.m, A.n, A.nnz, torch.cuda.get_device_name(A.val.device))


def csls_autotune(F, A, cache=None, stream=None):
    """Pick the SpMV threads-per-row for A x and A^T u by timing the candidates on
    this matrix (csls_autotune_spmv); with `cache` (a JSON path) the choice is
    looked up first and stored after tuning. Returns (group, group_t)."""
    import json
    key = _tune_key(A)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        g, gt = table[key]
        _check(_lib().csls_factor_set_spmv_groups(F.handle, int(g), int(gt)), "csls_factor_set_spmv_groups")
        return int(g), int(gt)
    work = _workspace(16 * (A.m + A.n) + 1024, A.val.device)
    g, gt = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * 2)()
    a = A.struct()
    _check(_lib().csls_autotune_spmv(F.handle, ctypes.byref(a), _ptr(work), work.numel(), ctypes.byref(g),
                                     ctypes.byref(gt), ms, _stream(stream)), "csls_autotune_spmv")
    if cache:
        table[key] = [g.value, gt.value]
        tmp = cache + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return g.value, gt.value


# --------------------------------------------------------------------------- autograd

class CslsSolve(torch.autograd.Function):
    """x = argmin ||A x - b|| with gradients for b and A's nonzero values."""

    @staticmethod
    def forward(ctx, val, b, row_ptr, col, m, n, opts_kw):
        A = Csr(row_ptr, col, val.detach(), m, n)
        F = csls_factor(A, **opts_kw)
        x, rep = csls_solve(F, A, b.detach(), **opts_kw)
        ctx.F, ctx.A, ctx.opts_kw = F, A, opts_kw
        ctx.save_for_backward(b.detach(), x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        b, x = ctx.saved_tensors
        gb, gv, _ = csls_solve_backward(ctx.F, ctx.A, b, x, grad_x.contiguous(), want_b=ctx.needs_input_grad[1],
                                        want_val=ctx.needs_input_grad[0], **ctx.opts_kw)
        return gv, gb, None, None, None, None, None


def solve(A, b, **opts_kw):
    """Differentiable solve for a torch sparse CSR tensor (or a Csr) and b."""
    if isinstance(A, Csr):
        return CslsSolve.apply(A.val, b, A.row_ptr, A.col, A.m, A.n, opts_kw)
    a = A.to_sparse_csr() if A.layout != torch.sparse_csr else A
    return CslsSolve.apply(a.values(), b, a.crow_indices(), a.col_indices().to(torch.int32), a.shape[0], a.shape[1],
                           opts_kw)
