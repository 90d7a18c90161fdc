"""The C ABI: libns.so builds, loads and exports every symbol include/ns.h declares.

These run without a GPU: no call here reaches a kernel (argument errors are
returned on the host before any launch).
"""
import ctypes
import os
import re

import pytest

from paper_2206_00975_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2206_00975_gb300 import build
    build.build()
    return _lib.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ns.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.ns_status_string(0) == b"NS_OK"
    assert lib.ns_status_string(4) == b"NS_ERR_NOCONV"
    assert b"sm_103a" in lib.ns_version()


def test_workspace_and_save_sizes(lib):
    d = _lib.SketchDesc(_lib.NS_SRHT, 8, 1024, 0, _lib.NS_PREC_FP64, 0)
    ws = lib.ns_workspace_size(ctypes.byref(d), 1 << 20, 256, 4)
    assert ws > 0 and ws % 256 == 0
    assert lib.ns_save_size(1024, 256) == 1024 * 256 + 256 * 256 + 256
    bad = _lib.SketchDesc(_lib.NS_SRHT, 8, 0, 0, _lib.NS_PREC_FP64, 0)
    assert lib.ns_workspace_size(ctypes.byref(bad), 100, 10, 1) == 0


def _desc(**kw):
    base = dict(kind=_lib.NS_SRHT, zeta=8, s=64, seed=1, prec=_lib.NS_PREC_FP64)
    base.update(kw)
    return _lib.SketchDesc(base["kind"], base["zeta"], base["s"], base["seed"], base["prec"], 0)


FAKE = ctypes.c_void_p(0x100000)   # never dereferenced: validation fails first


@pytest.mark.parametrize("kw,m,n,lda", [
    (dict(s=0), 100, 4, 100),             # s < 1
    (dict(s=256), 100, 4, 100),           # SRHT s > m' = 128
    (dict(), 100, 4, 99),                 # lda < m
    (dict(), 0, 4, 100),                  # m < 1
    (dict(kind=7), 100, 4, 100),          # unknown kind
    (dict(prec=9), 100, 4, 100),          # unknown precision
    (dict(kind=_lib.NS_SPARSE_SIGN, zeta=0), 100, 4, 100),
])
def test_sketch_rejects_bad_arguments(lib, kw, m, n, lda):
    d = _desc(**kw)
    st = lib.ns_sketch(ctypes.byref(d), FAKE, _lib.NS_F64, m, n, lda, FAKE, FAKE, 1 << 30, None)
    assert st == _lib.NS_ERR_INVALID_ARG


def test_solve_rejects_bad_k_and_short_workspace(lib):
    d = _desc(s=64)
    for k in (0, 5):
        st = lib.ns_solve(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, k, FAKE, FAKE, None, None, FAKE,
                          1 << 30, None)
        assert st == _lib.NS_ERR_INVALID_ARG
    st = lib.ns_solve(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, 1, FAKE, FAKE, None, None, FAKE, 16, None)
    assert st == _lib.NS_ERR_WORKSPACE
    # misaligned workspace
    st = lib.ns_solve(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, 1, FAKE, FAKE, None, None,
                      ctypes.c_void_p(0x100008), 1 << 30, None)
    assert st == _lib.NS_ERR_INVALID_ARG


def test_null_pointers_rejected(lib):
    d = _desc()
    assert lib.ns_sketch(ctypes.byref(d), None, _lib.NS_F64, 100, 4, 100, FAKE, FAKE, 1 << 30, None) == \
        _lib.NS_ERR_INVALID_ARG
    assert lib.ns_sketch(None, FAKE, _lib.NS_F64, 100, 4, 100, FAKE, FAKE, 1 << 30, None) == _lib.NS_ERR_INVALID_ARG


def test_solve_eps_rejects_bad_tolerance(lib):
    d = _desc(s=64)
    for eps in (-1.0, float("nan")):
        st = lib.ns_solve_eps(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, eps, FAKE, FAKE, FAKE, None, None,
                              FAKE, 1 << 30, None)
        assert st == _lib.NS_ERR_INVALID_ARG
    # a missing k output
    st = lib.ns_solve_eps(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, 1e-8, FAKE, FAKE, None, None, None,
                          FAKE, 1 << 30, None)
    assert st == _lib.NS_ERR_INVALID_ARG


def test_sketch_update_rejects_bad_arguments(lib):
    d = _desc(s=64)
    for m0, op, j in ((100, 2, 5), (100, 0, 50), (0, 1, 0), (100, 1, -1)):
        assert lib.ns_sketch_update(ctypes.byref(d), m0, op, j, FAKE, 4, FAKE, None) == _lib.NS_ERR_INVALID_ARG
    assert lib.ns_sketch_update(ctypes.byref(d), 100, 1, 5, None, 4, FAKE, None) == _lib.NS_ERR_INVALID_ARG


def test_hrht_rejections(lib):
    d = _desc(kind=_lib.NS_HRHT, s=256)
    # s > m' = 128
    assert lib.ns_sketch(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, FAKE, FAKE, 1 << 30, None) == \
        _lib.NS_ERR_INVALID_ARG
    d = _desc(kind=_lib.NS_HRHT, s=64)
    # m' > 2^24, FP32 input, FP32-stream precision
    assert lib.ns_sketch(ctypes.byref(d), FAKE, _lib.NS_F64, (1 << 24) + 1, 1, (1 << 24) + 1, FAKE, FAKE, 1 << 40,
                         None) == _lib.NS_ERR_INVALID_ARG
    assert lib.ns_sketch(ctypes.byref(d), FAKE, _lib.NS_F32, 100, 4, 100, FAKE, FAKE, 1 << 30, None) == \
        _lib.NS_ERR_INVALID_ARG
    d32 = _desc(kind=_lib.NS_HRHT, s=64, prec=_lib.NS_PREC_FP32_STREAM)
    assert lib.ns_sketch(ctypes.byref(d32), FAKE, _lib.NS_F32, 100, 4, 100, FAKE, FAKE, 1 << 30, None) == \
        _lib.NS_ERR_INVALID_ARG
    # row updates take O(s) columns of S; the H-RHT's takes all m' coordinates
    assert lib.ns_sketch_update(ctypes.byref(d), 100, 1, 5, FAKE, 4, FAKE, None) == _lib.NS_ERR_INVALID_ARG
    # the workspace holds the transformed blocks: at least 8 m' n bytes
    assert lib.ns_workspace_size(ctypes.byref(d), 1 << 20, 256, 4) >= 8 * (1 << 20) * 256
