"""The allocation-free sketch entry point.

csls_sketch_noalloc serves callers that cannot call cudaMalloc themselves (for
example code whose device memory is owned by another framework's pool
allocator): it takes its scratch from a fixed 16 MiB array inside the library
instead of a caller workspace. Its output must equal csls_sketch's on the same
input, including on a second call right after the first (the shared scratch
keeps the previous call's contents, which the call must clear), and sizes
beyond the fixed maximum must be refused before any device work.
"""
import ctypes

import numpy as np
import pytest
import torch

from workloads import config_problem, poisson2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csls():
    from paper_2409_15818_gb300 import build
    build.build()
    from paper_2409_15818_gb300 import csls as mod
    return mod


def _dev(csls, p):
    return csls.Csr.from_numpy(p.row_ptr, p.col, p.val, p.m, p.n)


def _as_sa(t, s):
    torch.cuda.synchronize()
    return t.cpu().numpy().T[:s, :]


def test_noalloc_sketch_matches_workspace_sketch_twice(csls):
    cases = [(config_problem("cfg1"), 1600, 11, "f64"), (poisson2d(3, 2, 37, 11, 9, R=1.5, seed=7), 301, 5, "f64"),
             (config_problem("cfg1"), 977, 3, "f32")]
    for p, s, seed, prec in cases:   # consecutive calls share the static scratch
        A = _dev(csls, p)
        got, status = csls.csls_sketch_noalloc(A, s, seed, prec=prec)
        assert status == 0
        want = csls.csls_sketch(A, s, seed, prec=prec)
        g, w = _as_sa(got, s), _as_sa(want, s)
        assert np.array_equal(np.ascontiguousarray(g).view(np.uint8), np.ascontiguousarray(w).view(np.uint8))


def test_noalloc_rejects_sizes_beyond_the_static_scratch(csls):
    p = config_problem("cfg1")
    A = _dev(csls, p)
    s = 1 << 22   # needs about 16 s = 64 MiB of scratch
    SA = torch.empty(8, dtype=torch.float64, device="cuda")   # never touched: refused on the host
    a = A.struct()
    st = csls._lib().csls_sketch_noalloc(ctypes.byref(a), s, 1, 0, ctypes.c_void_p(SA.data_ptr()), s,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 9   # CSLS_ERR_WORKSPACE
