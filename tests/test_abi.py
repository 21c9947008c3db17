"""The C-ABI library loads and exports every entry point include/radgeb.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "radgeb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rg_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2511_04277_gb300 as pkg
    path = pkg.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rg_create", "rg_trace", "rg_counts_to_F", "rg_enforce_iterative", "rg_enforce_lsq",
                 "rg_aggregate", "rg_gebhart", "rg_gebhart_adjoint", "rg_temperatures",
                 "rg_temperatures_adjoint"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2511_04277_gb300 import _native
    assert sorted(_native.SIGNATURES) == _declared()


def test_version_string(lib):
    lib.rg_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rg_version()


def test_create_reports_no_device_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.rg_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    st = lib.rg_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value


def _declarations():
    """name -> list of parameter type strings, from the header's prototypes."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    text = re.sub(r"#.*", "", text)
    out = {}
    for m in re.finditer(r"\b(rg_[A-Za-z_0-9]+)\s*\(([^;{()]*)\)\s*;", text):
        params = [p.strip() for p in m.group(2).split(",") if p.strip()]
        if params == ["void"]:
            params = []
        out[m.group(1)] = params
    return out


def _kind_of_c(param):
    """The calling-convention class of a C parameter: pointer, 64-bit or 32-bit integer,
    double or float."""
    if "*" in param:
        return "ptr"
    t = param.rsplit(None, 1)[0].replace("const", "").strip()
    return {"int64_t": "i64", "uint64_t": "i64", "size_t": "i64", "int32_t": "i32", "uint32_t": "i32", "int": "i32",
            "double": "f64", "float": "f32"}[t]


def _kind_of_ctypes(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    return {ctypes.c_int64: "i64", ctypes.c_uint64: "i64", ctypes.c_int32: "i32", ctypes.c_uint32: "i32",
            ctypes.c_double: "f64", ctypes.c_float: "f32"}[t]


def test_binding_argument_types_match_the_header():
    """Every ctypes signature has the header prototype's parameter count and, parameter
    by parameter, its class (pointer / 64-bit / 32-bit integer / double / float): a
    mismatch would pass a wrong-sized argument without any error."""
    from paper_2511_04277_gb300 import _native
    decl = _declarations()
    assert sorted(decl) == sorted(_native.SIGNATURES)
    for name, params in decl.items():
        argtypes = _native.SIGNATURES[name][1]
        assert len(argtypes) == len(params), (name, params, argtypes)
        for p, a in zip(params, argtypes):
            assert _kind_of_c(p) == _kind_of_ctypes(a), (name, p, a)


def test_solver_workspace_sizes_without_a_gpu():
    """The caller-owned workspace sizes are pure host arithmetic: positive, growing with n,
    the REF query equal to rg_solver_workspace's, the factor store a header, one 16-bit np x np
    block and one fp64 scale vector of np per set."""
    from paper_2511_04277_gb300 import api
    from paper_2511_04277_gb300._native import RadgebError
    for kind in ("gebhart", "gebhart_adjoint", "temperatures", "temperatures_sets", "enforce_lsq"):
        a, b = api.solver_workspace(kind, 300), api.solver_workspace(kind, 1000)
        assert 0 < a < b, kind
    assert api.solver_workspace("gebhart_adjoint_factored", 500, 2) > 0
    assert api.gebhart_workspace(700, 3, "fp16") == api.solver_workspace("gebhart", 700)
    # the adjoint keeps F^T Lambda as well: more than the forward solve
    assert api.solver_workspace("gebhart_adjoint", 700) > api.solver_workspace("gebhart", 700)
    assert api.gebhart_workspace(700, 3, "bf16", keep_factors=True) == 256 + 3 * 768 * 768 * 2 + 3 * 768 * 8
    with pytest.raises(RadgebError):
        api.gebhart_workspace(0, 1, "bf16", keep_factors=True)
    with pytest.raises(RadgebError):
        api.solver_workspace("enforce_lsq", 5000)
