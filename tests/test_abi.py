"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every function include/gk.h declares, and its argument checks answer before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgk():
    from paper_2006_16852_gb300 import build
    build.build()
    import paper_2006_16852_gb300 as gk
    return gk.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"GK_API\s+[\w\s\*]+?\b(gk_\w+)\s*\(", text))
    return names


def test_header_declares_the_paper_calls():
    d = _declared()
    for name in ("gk_apply", "gk_apply_adv", "gk_solver_generate", "gk_solve", "gk_precond_generate"):
        assert name in d


def test_every_declared_symbol_is_exported(libgk):
    import paper_2006_16852_gb300 as gk
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(libgk, name), f"{name} not exported"
    assert declared <= set(gk.EXPORTS)


def test_version_and_error_string(libgk):
    assert libgk.gk_version() >= 100
    assert isinstance(libgk.gk_last_error(), bytes)


def test_argument_errors_without_device(libgk):
    out = ctypes.c_void_p()
    rc = libgk.gk_matrix_create_csr(-1, 1, 0, None, None, None, 0, 0, None, ctypes.byref(out))
    assert rc == 1 and b"negative" in libgk.gk_last_error()
    rc = libgk.gk_matrix_create_csr(1, 1, 0, None, None, None, 0, 0, None, None)
    assert rc == 1
    rc = libgk.gk_matrix_create_csr(1, 1, 0, ctypes.c_void_p(8), None, None, 1, 0, None, ctypes.byref(out))
    assert rc == 8  # FP32 storage is not built
    rc = libgk.gk_matrix_create_csr(1, 1, 0, ctypes.c_void_p(8), None, None, 7, 0, None, ctypes.byref(out))
    assert rc == 3
    rc = libgk.gk_matrix_create_csr(1, 1, 0, ctypes.c_void_p(8), None, None, 0, 9, None, ctypes.byref(out))
    assert rc == 1
    assert libgk.gk_apply(None, None, None, None) == 1
    assert libgk.gk_solve(None, None, None, None, None) == 1
    assert libgk.gk_matrix_destroy(None) == 1
    assert libgk.gk_dot(-1, None, None, None, None) == 1
    assert libgk.gk_wait_selftest(None, None) == 1
