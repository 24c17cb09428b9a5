"""The C ABI without a GPU: symbols, host-only calls, argument errors.

The library must load and export every function include/sm.h declares. The
host-only entry points (comparison orders) are checked against the oracle,
and argument validation is checked on calls that fail before any device
work.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1612_01506_gb300 import sm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return sm.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sm_[a-z_0-9]+)\s*\(", src)))


def test_header_matches_binding():
    assert declared_functions() == sorted(sm.EXPORTS)


def test_exports(lib):
    out = os.popen(f"nm -D --defined-only {sm.library_path()}").read()
    exported = set(re.findall(r"\bT (sm_[a-z_0-9]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_status_strings(lib):
    for code, name in enumerate(["SM_OK", "SM_EINVAL", "SM_ENOMEM", "SM_ECUDA", "SM_ETRUNC", "SM_ETIMEOUT",
                                 "SM_ENOTSUP"]):
        assert lib.sm_status_string(code).decode() == name


def test_order_matches_oracle(lib, orc):
    r = np.random.default_rng(3)
    for m in (1, 2, 3, 17, 64, 1000, 4096):
        hist = r.integers(0, 40, size=256).astype(np.uint64)
        p = r.integers(0, 256, size=m, dtype=np.uint8)
        assert np.array_equal(sm.sm_order(p, hist), orc.order_freq(p, hist))
        assert np.array_equal(sm.sm_order_fixed(p, sm.SM_ORDER_H), orc.order_h(m))
        ps = r.choice(np.frombuffer(b"ab  cd", np.uint8), size=m)
        assert np.array_equal(sm.sm_order_fixed(ps, sm.SM_ORDER_HS), orc.order_hs(ps))


def test_host_argument_errors(lib):
    h = np.zeros(256, dtype=np.uint64)
    pi = np.zeros(4, dtype=np.uint32)
    u64p, u32p = C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)
    pat = (C.c_uint8 * 4)(*b"abcd")
    assert lib.sm_order(pat, 0, h.ctypes.data_as(u64p), pi.ctypes.data_as(u32p)) == sm.SM_EINVAL
    assert lib.sm_order(None, 4, h.ctypes.data_as(u64p), pi.ctypes.data_as(u32p)) == sm.SM_EINVAL
    assert lib.sm_order_fixed(pat, 4, 7, pi.ctypes.data_as(u32p)) == sm.SM_EINVAL
    assert lib.sm_order_fixed(None, 4, sm.SM_ORDER_HS, pi.ctypes.data_as(u32p)) == sm.SM_EINVAL
    assert lib.sm_count(None, None, 0, pat, 4, None, None, None) == sm.SM_EINVAL
    assert lib.sm_report(None, None, 0, pat, 4, None, None, 0, None, None) == sm.SM_EINVAL
    assert lib.sm_histogram(None, None, 0, None, None) == sm.SM_EINVAL
    assert lib.sm_sync(None, None) == sm.SM_EINVAL
    assert lib.sm_set_knob(None, 1, 4) == sm.SM_EINVAL
    assert b"NULL" in lib.sm_last_error()
    lib.sm_destroy(None)


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.sm_create(C.byref(h), 0)
    assert st in (sm.SM_ECUDA, sm.SM_EINVAL) and not h.value
    assert lib.sm_last_error()


def test_product_path_has_no_oracle_dependency():
    # the package and the CUDA sources never import, include or link the oracle
    pkg = os.path.join(ROOT, "paper_1612_01506_gb300")
    for dirpath, _dirs, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle|#include .*oracle)", text, flags=re.M), f
