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


INV, WSP = _lib.NS_ERR_INVALID_ARG, 2  # NS_ERR_WORKSPACE
MIS = ctypes.c_void_p(0x100008)        # not 256-byte aligned


def test_solve_sketched_and_stats_rejections(lib):
    d = _desc(s=64)
    for n, k in ((4, 0), (4, 5), (65, 1), (0, 1)):  # k outside 1..n, n > s, n < 1
        assert lib.ns_solve_sketched(ctypes.byref(d), FAKE, n, k, FAKE, FAKE, None, None, FAKE, 1 << 30,
                                     None) == INV
    assert lib.ns_solve_sketched(ctypes.byref(d), None, 4, 1, FAKE, FAKE, None, None, FAKE, 1 << 30, None) == INV
    assert lib.ns_solve_sketched(ctypes.byref(d), FAKE, 4, 1, FAKE, FAKE, None, None, MIS, 1 << 30, None) == INV
    assert lib.ns_solve_sketched(ctypes.byref(d), FAKE, 4, 1, FAKE, FAKE, None, None, FAKE, 16, None) == WSP
    assert lib.ns_solve_stats(ctypes.byref(d), 0, 4, FAKE, FAKE, None) == INV
    assert lib.ns_solve_stats(ctypes.byref(d), 100, 5000, FAKE, FAKE, None) == INV
    assert lib.ns_solve_stats(ctypes.byref(d), 100, 4, None, FAKE, None) == INV
    assert lib.ns_sketched_stats(ctypes.byref(d), 0, FAKE, FAKE, None) == INV
    assert lib.ns_sketched_stats(ctypes.byref(d), 4, FAKE, None, None) == INV


def test_backward_rejections(lib):
    d = _desc(s=64)
    bw = lambda dd, m, n, k, ldd, ws=FAKE, nb=1 << 30: lib.ns_backward(  # noqa: E731
        ctypes.byref(dd), m, n, k, FAKE, FAKE, FAKE, FAKE, ldd, ws, nb, None)
    assert bw(_desc(s=64, kind=_lib.NS_SPARSE_SIGN), 100, 4, 1, 100) == INV  # SRHT only
    assert bw(_desc(s=64, kind=_lib.NS_HRHT), 100, 4, 1, 100) == INV
    assert bw(d, 100, 4, 4, 100) == INV      # k >= n (the projector has no complement)
    assert bw(d, 100, 1, 1, 100) == INV      # n < 2
    assert bw(d, 100, 4, 1, 99) == INV       # ldd < m
    assert bw(_desc(s=256), 100, 4, 1, 100) == INV  # s > m'
    assert bw(d, 100, 4, 1, 100, ws=MIS) == INV
    assert bw(d, 100, 4, 1, 100, nb=16) == WSP


def _problem(**kw):
    base = dict(A=0x100000, m=1000, n=8, lda=1000, s=32, k=1, tls=0, seed=1, Vk=0x100000, sigk=0x100000, x=0,
                dtype=_lib.NS_F64, reserved=0)
    base.update(kw)
    return _lib.Problem(**base)


def test_batched_rejections(lib):
    d = _desc()
    ok = (_lib.Problem * 1)(_problem())
    assert lib.ns_batched_workspace_size(ctypes.byref(d), 1, ok) > 0
    for bad in (dict(s=4), dict(s=2048), dict(m=4), dict(lda=999), dict(k=0), dict(k=9), dict(tls=1),
                dict(tls=1, k=1, x=0), dict(A=0x100004), dict(A=0), dict(Vk=0), dict(dtype=2),
                dict(dtype=_lib.NS_F32, A=0x100002)):
        arr = (_lib.Problem * 2)(_problem(), _problem(**bad))
        assert lib.ns_batched_workspace_size(ctypes.byref(d), 2, arr) == 0, bad
        assert lib.ns_solve_batched(ctypes.byref(d), 2, arr, FAKE, FAKE, FAKE, 1 << 30, None) == INV, bad
    dsp = _desc(kind=_lib.NS_SPARSE_SIGN)
    assert lib.ns_batched_workspace_size(ctypes.byref(dsp), 1, ok) == 0
    assert lib.ns_solve_batched(ctypes.byref(dsp), 1, ok, FAKE, FAKE, FAKE, 1 << 30, None) == INV
    assert lib.ns_solve_batched(ctypes.byref(d), 0, ok, FAKE, FAKE, FAKE, 1 << 30, None) == INV
    assert lib.ns_solve_batched(ctypes.byref(d), 1, ok, FAKE, FAKE, MIS, 1 << 30, None) == INV
    assert lib.ns_solve_batched(ctypes.byref(d), 1, ok, FAKE, FAKE, FAKE, 16, None) == WSP


def test_aaa_rejections(lib):
    d = _desc(s=400)
    assert lib.ns_aaa_workspace_size(ctypes.byref(d), 1 << 17, 100) > 0
    assert lib.ns_aaa_workspace_size(ctypes.byref(d), 1, 100) == 0          # m < 2
    assert lib.ns_aaa_workspace_size(ctypes.byref(d), 1 << 17, 401) == 0    # K > s
    assert lib.ns_aaa_workspace_size(ctypes.byref(d), 200, 100) == 0        # s > m' = 256
    assert lib.ns_aaa_workspace_size(ctypes.byref(_desc(s=400, kind=_lib.NS_HRHT)), 1 << 17, 100) == 0
    aaa = lambda x=FAKE, ws=FAKE, nb=1 << 30: lib.ns_aaa_real(  # noqa: E731
        ctypes.byref(d), x, FAKE, 1 << 17, 100, None, FAKE, FAKE, FAKE, None, FAKE, ws, nb, None)
    assert aaa(x=None) == INV
    assert aaa(ws=MIS) == INV
    assert aaa(nb=16) == WSP


def test_residual_and_meta_rejections(lib):
    res = lambda dtype=_lib.NS_F64, m=100, n=4, lda=100, k=1, nb=1 << 20: lib.ns_residual(  # noqa: E731
        FAKE, dtype, m, n, lda, FAKE, k, FAKE, FAKE, nb, None)
    assert res(dtype=_lib.NS_F32) == INV
    for k in (0, 17):
        assert res(k=k) == INV
    assert res(lda=99) == INV
    assert res(nb=16) == WSP
    assert res(n=4096, k=16) == INV          # W would not fit in shared memory
    d = _desc(s=64)
    assert lib.ns_srht_meta(ctypes.byref(_desc(s=64, kind=_lib.NS_SPARSE_SIGN)), 100, FAKE, FAKE, None) == INV
    assert lib.ns_srht_meta(ctypes.byref(_desc(s=256)), 100, FAKE, FAKE, None) == INV
    assert lib.ns_srht_meta(ctypes.byref(d), 0, FAKE, FAKE, None) == INV
    assert lib.ns_sparse_meta(ctypes.byref(d), 100, FAKE, FAKE, None) == INV   # not sparse-sign
    dsp = _desc(s=64, kind=_lib.NS_SPARSE_SIGN)
    assert lib.ns_sparse_meta(ctypes.byref(dsp), 100, None, FAKE, None) == INV


def test_sketch_static_rejections(lib):
    st = lambda dd, dtype=_lib.NS_F64, m=100, lda=100, A=FAKE: lib.ns_sketch_static(  # noqa: E731
        ctypes.byref(dd), A, dtype, m, 4, lda, FAKE, None, None)
    assert st(_desc(kind=_lib.NS_HRHT)) == INV
    assert st(_desc(kind=_lib.NS_SPARSE_SIGN)) == INV
    assert st(_desc(), dtype=_lib.NS_F32) == INV
    assert st(_desc(s=256)) == INV            # s > m'
    assert st(_desc(), lda=99) == INV
    assert st(_desc(), A=ctypes.c_void_p(0x100004)) == INV
    assert st(_desc(s=1024), m=1 << 24, lda=1 << 24) == WSP  # scratch above the static 16 MiB


def test_bounded_wait_hook_rejections(lib):
    hook = lambda which=0, limit=100, status=FAKE, ws=ctypes.c_void_p(0x100000), nb=256: \
        lib.ns_test_bounded_wait(which, limit, status, ws, nb, None)  # noqa: E731
    assert hook(which=2) == INV
    assert hook(limit=0) == INV
    assert hook(limit=(1 << 24) + 1) == INV
    assert hook(status=None) == INV
    assert hook(ws=None) == INV            # the grid-barrier form needs a word of scratch
    assert hook(ws=MIS) == INV
    assert hook(nb=128) == INV


def test_sweep_limit_range(lib):
    # the descriptor's Jacobi sweep limit: 0 (default 30) .. 30
    for bad in (-1, 31):
        d = _lib.SketchDesc(_lib.NS_SRHT, 8, 64, 1, _lib.NS_PREC_FP64, bad)
        assert lib.ns_workspace_size(ctypes.byref(d), 100, 4, 1) == 0
        st = lib.ns_solve(ctypes.byref(d), FAKE, _lib.NS_F64, 100, 4, 100, 1, FAKE, FAKE, None, None, FAKE,
                          1 << 30, None)
        assert st == INV
    d = _lib.SketchDesc(_lib.NS_SRHT, 8, 64, 1, _lib.NS_PREC_FP64, 1)
    assert lib.ns_workspace_size(ctypes.byref(d), 100, 4, 1) > 0


def test_batched_fp32_problems_and_tuning(lib):
    d32 = _lib.SketchDesc(_lib.NS_SRHT, 8, 32, 0, _lib.NS_PREC_FP32_STREAM, 0)
    ok32 = (_lib.Problem * 1)(_problem(dtype=_lib.NS_F32, A=0x100004))  # 4-byte alignment suffices for FP32
    assert lib.ns_batched_workspace_size(ctypes.byref(d32), 1, ok32) > 0
    dg = _lib.SketchDesc(_lib.NS_GAUSSIAN, 8, 32, 0, _lib.NS_PREC_BF16X3, 0)
    assert lib.ns_batched_workspace_size(ctypes.byref(dg), 1, ok32) == 0
    assert lib.ns_batched_tuning(2, 4, 1) == 0
    assert lib.ns_batched_tuning(0, 0, 0) == 0   # back to the defaults
    for bad in ((-1, 0, 0), (65, 0, 0), (1, -2, 0), (1, 0, 99)):
        assert lib.ns_batched_tuning(*bad) == INV


def test_sketch_rows_rejections(lib):
    rows = lambda dd, m_total=1000, o=0, m_p=100, lda=100, A=FAKE, nb=1 << 30: lib.ns_sketch_rows(  # noqa: E731
        ctypes.byref(dd), A, _lib.NS_F64, m_total, o, m_p, 4, lda, FAKE, None, FAKE, nb, None)
    d = _desc(s=64)
    assert lib.ns_sketch_rows_workspace_size(ctypes.byref(d), 1000, 0, 100, 4) > 0
    assert rows(d, o=950) == INV                      # beyond m_total
    assert rows(d, o=-1) == INV
    assert rows(d, m_p=0) == INV
    assert rows(d, lda=99) == INV
    assert rows(_desc(s=64, kind=_lib.NS_HRHT)) == INV
    assert rows(_desc(s=64, kind=_lib.NS_GAUSSIAN, prec=_lib.NS_PREC_BF16X3)) == INV
    assert rows(_desc(s=2048)) == INV                 # SRHT s > m' = 1024
    assert rows(d, nb=16) == WSP


def test_solve_pipelined_rejections(lib):
    d = _desc(s=64)
    ptrs = (ctypes.c_void_p * 2)(0x100000, 0x200000)
    call = lambda dd=d, A=ptrs, count=2, m=100, n=4, lda=100, k=1, nb=1 << 30: lib.ns_solve_pipelined(  # noqa: E731
        ctypes.byref(dd), A, count, _lib.NS_F64, m, n, lda, k, FAKE, FAKE, None, FAKE, nb, None)
    assert lib.ns_solve_pipelined_workspace_size(ctypes.byref(d), 100, 4) > \
        lib.ns_workspace_size(ctypes.byref(d), 100, 4, 1) // 2
    assert call(count=0) == INV
    assert call(A=None) == INV
    assert call(A=(ctypes.c_void_p * 2)(0x100000, 0)) == INV         # a null problem
    assert call(A=(ctypes.c_void_p * 2)(0x100000, 0x100004)) == INV  # a misaligned problem
    assert call(k=0) == INV
    assert call(k=5) == INV
    assert call(lda=99) == INV
    assert call(nb=16) == WSP
