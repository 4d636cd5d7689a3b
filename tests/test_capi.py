"""CPU-side checks of the C ABI: the library builds, loads, and exports every
symbol the header declares; host-side validation paths that need no GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nrd.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int)\s+(nrd_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1302_6303_gb300 import nrd
    return nrd.load()


def test_header_declares_expected_calls():
    syms = declared_symbols()
    for s in ["nrd_create", "nrd_set_hierarchy", "nrd_residual", "nrd_jv", "nrd_precond_apply",
              "nrd_newton", "nrd_step", "nrd_tag"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    from paper_1302_6303_gb300 import nrd
    assert sorted(nrd.EXPORTED) == declared_symbols()


def test_params_default_and_create_without_gpu(lib):
    import ctypes
    from paper_1302_6303_gb300 import nrd
    p = nrd.Params()
    assert lib.nrd_params_default(ctypes.byref(p)) == 0
    assert p.k == 0.01 and p.u_min == 1e-6 and p.restart == 30
    assert lib.nrd_params_default(None) == nrd.EINVAL
    bad = nrd.Params()
    lib.nrd_params_default(ctypes.byref(bad))
    bad.restart = 0
    h = ctypes.c_void_p()
    assert lib.nrd_create(ctypes.byref(bad), ctypes.byref(h)) == nrd.EINVAL
    assert lib.nrd_create(ctypes.byref(p), ctypes.byref(h)) == 0
    assert lib.nrd_last_error(None) == b"null context"
    assert lib.nrd_residual(h, None, None, 1.0, 1.0, None, None) == nrd.ESTATE
    assert lib.nrd_destroy(h) == 0
    assert lib.nrd_destroy(None) == nrd.EINVAL


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_1302_6303_gb300 import nrd
    saved = nrd._lib
    try:
        nrd._lib = None
        with pytest.raises(RuntimeError):
            nrd.load(str(tmp_path / "missing.so"))
    finally:
        nrd._lib = saved
