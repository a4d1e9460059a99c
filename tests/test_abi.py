"""The C-ABI library builds, loads and exports every symbol include/cat.h declares;
host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

from paper_2406_17284_gb300 import build as cat_build
from paper_2406_17284_gb300 import cat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^CAT_API\s+[\w\s\*]*?\b(cat_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    cat_build.build()
    return cat.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(cat.EXPORTED)


def test_version(lib):
    assert "sm_103a" in cat.cat_version()


def test_create_rejects_bad_arguments_without_gpu(lib):
    good = cat.make_rule(1, 2, 0, 2, 3, 3, 3)
    out = ctypes.c_void_p()
    cases = [
        (0, 10, good, 0, cat.CAT_ERR_INVALID_ARG),
        (10, 0, good, 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, cat.make_rule(0, 2, 0, 2, 3, 3, 3), 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, cat.make_rule(33, 2, 0, 2, 3, 3, 3), 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, cat.make_rule(17, 2, 0, 2, 3, 3, 3), 1, cat.CAT_ERR_UNSUPPORTED),   # r > 16: zero boundary only
        (10, 10, cat.make_rule(1, 1, 0, 2, 3, 3, 3), 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, cat.make_rule(1, 2, 2, 2, 3, 3, 3), 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, cat.make_rule(1, 2, 0, -1, 3, 3, 3), 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, cat.make_rule(1, 2, 0, 2, 3, 3, 3, nbhd="X"), 0, cat.CAT_ERR_INVALID_ARG),
        (10, 10, good, -1, cat.CAT_ERR_INVALID_ARG),   # boundaries: 0 zero, 1 periodic
        (10, 10, good, 7, cat.CAT_ERR_INVALID_ARG),
        (1 << 40, 1 << 20, good, 0, cat.CAT_ERR_INVALID_ARG),
    ]
    for H, W, rule, b, want in cases:
        rc = lib.cat_create(H, W, ctypes.byref(rule), b, ctypes.byref(out))
        assert rc == want, (H, W, b, rc, lib.cat_last_error())
        assert out.value is None
        assert lib.cat_last_error()
    # one-bit storage: two-state Moore rules with the zero boundary; unknown storage codes
    vn = cat.make_rule(1, 2, 0, 2, 3, 3, 3, nbhd="N")
    multi = cat.make_rule(1, 3, 0, 2, 3, 3, 3)
    for rule, b, st, want in [(vn, 0, cat.STORE_BIT1, cat.CAT_ERR_UNSUPPORTED),
                              (multi, 0, cat.STORE_BIT1, cat.CAT_ERR_UNSUPPORTED),
                              (good, 1, cat.STORE_BIT1, cat.CAT_ERR_UNSUPPORTED),
                              (good, 0, 5, cat.CAT_ERR_INVALID_ARG)]:
        rc = lib.cat_create_ex(10, 10, ctypes.byref(rule), b, st, ctypes.byref(out))
        assert rc == want, (rule.nbhd, b, st, rc, lib.cat_last_error())
        assert out.value is None


def test_null_handles_rejected(lib):
    assert lib.cat_step(None, 1, None) == cat.CAT_ERR_INVALID_ARG
    assert lib.cat_set_options(None, 0, 0, 0, 1) == cat.CAT_ERR_INVALID_ARG
    assert lib.cat_status(None, None) == cat.CAT_ERR_INVALID_ARG
    assert lib.cat_destroy(None) == cat.CAT_OK
    assert lib.cat_batch_step(None, 1, 1, None) == cat.CAT_ERR_INVALID_ARG
    assert lib.cat_bind(None, None, None, 16) == cat.CAT_ERR_INVALID_ARG


def test_tensor_probe_rejects_bad_arguments_without_gpu(lib):
    assert lib.cat_tensor_probe(cat.DTYPE_INT8, 16, 1024, None) == cat.CAT_ERR_UNSUPPORTED
    assert lib.cat_tensor_probe(cat.DTYPE_FP8_E4M3, 0, 1024, None) == cat.CAT_ERR_INVALID_ARG
    assert lib.cat_tensor_probe(cat.DTYPE_FP16, 16, None, None) == cat.CAT_ERR_INVALID_ARG
    assert b"d_status" in lib.cat_last_error()
