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
