"""CPU-side checks of the CUDA library: it builds, loads and exports every
entry point that include/csls.h declares (no compute without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "csls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(csls_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_15818_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("csls_sketch", "csls_factor", "csls_solve", "csls_solve_backward", "csls_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2409_15818_gb300 import csls
    assert set(_declared()) <= set(csls.EXPORTS)


def test_status_strings_and_defaults(lib):
    from paper_2409_15818_gb300 import csls
    for code in range(10):
        assert csls.csls_status_string(code).startswith("CSLS_")
    o = csls.make_opts()
    assert o.gamma == 4.0 and o.atol == 1e-12 and o.guard_cond == 10.0 and o.spin_limit > 0


def test_argument_errors_without_gpu(lib):
    """Size and pointer checks run on the host before any device work."""
    from paper_2409_15818_gb300 import csls
    L = csls._lib()
    bad = csls.csls_csr(0, 5, 0, 0, 0, 0)
    nbytes = ctypes.c_size_t()
    assert L.csls_sketch_workspace(ctypes.byref(bad), 4, ctypes.byref(nbytes)) == 1
    A = csls.csls_csr(10, 20, 0, 8, 0, 0)   # m < n: no full column rank
    o = csls.make_opts()
    pb, tb = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.csls_factor_workspace(ctypes.byref(A), ctypes.byref(o), ctypes.byref(pb), ctypes.byref(tb)) == 1
    ok = csls.csls_csr(100, 10, 0, 8, 0, 0)
    assert L.csls_factor_workspace(ctypes.byref(ok), ctypes.byref(o), ctypes.byref(pb), ctypes.byref(tb)) == 0
    assert pb.value > 10 * 10 * 8 and tb.value > 40 * 10 * 8


def _prototypes():
    """name -> (return type text, parameter list) for every function csls.h declares."""
    src = open(os.path.join(ROOT, "include", "csls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#.*", "", src)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(csls_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        params = " ".join(params.split())
        plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        out[name] = (" ".join(ret.split()), plist)
    return out


def test_binding_signatures_match_the_header():
    """Each ctypes prototype has the header's parameter count, and pointer, double and integer-width kinds line up."""
    from paper_2409_15818_gb300 import csls
    protos = _prototypes()
    assert set(protos) == set(_declared())

    def kind_of_c(t):
        t = t.replace("const ", "")
        if "*" in t or t.startswith("csls_stream_t"):
            return "ptr"
        if t.startswith("double"):
            return "double"
        if t.startswith(("int64_t", "uint64_t", "size_t")):
            return "int8B"
        if t.startswith(("int ", "int32_t", "uint32_t")):
            return "int4B"
        raise AssertionError("unclassified parameter type: " + t)

    def kind_of_ctypes(c):
        if c in (ctypes.c_void_p, ctypes.c_char_p):
            return "ptr"
        if c is ctypes.c_double:
            return "double"
        return "int%dB" % ctypes.sizeof(c)

    for name, (ret, params) in protos.items():
        res, args = csls.EXPORTS[name]
        assert len(args) == len(params), (name, len(args), params)
        for c_type, a in zip(params, args):
            assert kind_of_ctypes(a) == kind_of_c(c_type), (name, c_type, a)
        if ret == "void":
            assert res is None, name
        elif "char" in ret:
            assert res is ctypes.c_char_p, name
        else:
            assert res is ctypes.c_int, (name, ret)
