"""Python binding of libns with the C ABI's names (include/ns.h).

Tensors are torch CUDA tensors; matrices are column-major, i.e. a tensor of
shape (rows, cols) with stride (1, ld).  ``colmajor(x)`` makes such a copy.
These wrappers only marshal arguments: they allocate outputs and the
workspace with torch, pass raw pointers and the current CUDA stream, and
raise NSError on a non-OK status.
"""
import ctypes

import torch

from . import _lib
from ._lib import Problem  # noqa: F401
from ._lib import (NS_F32, NS_F64, NS_GAUSSIAN, NS_HRHT, NS_PREC_BF16X3, NS_PREC_FP32_STREAM, NS_PREC_FP64,  # noqa: F401
                   NS_ROW_APPEND, NS_ROW_REMOVE, NS_SPARSE_SIGN, NS_SRHT, NSError, SketchDesc)


def desc(kind=NS_SRHT, s=0, seed=0, zeta=8, prec=NS_PREC_FP64, max_sweeps=0):
    return SketchDesc(int(kind), int(zeta), int(s), int(seed) & ((1 << 64) - 1), int(prec), int(max_sweeps))


def colmajor(x, dtype=None, device=None):
    """Copy of a 2-D array/tensor as a column-major torch tensor (stride (1, rows))."""
    t = torch.as_tensor(x)
    if dtype is not None:
        t = t.to(dtype)
    if device is not None:
        t = t.to(device)
    return t.t().contiguous().t()


def _ld(A):
    if A.dim() != 2 or A.stride(0) != 1:
        raise ValueError("expected a column-major matrix (stride (1, ld))")
    return max(A.stride(1), A.shape[0]) if A.shape[1] > 1 else max(A.shape[0], 1)


def _dtype_code(A):
    if A.dtype == torch.float64:
        return NS_F64
    if A.dtype == torch.float32:
        return NS_F32
    raise ValueError("A must be float64 or float32")


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _empty_cm(rows, cols, device, dtype=torch.float64):
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def workspace_size(d, m, n, k=1):
    return int(_lib.load().ns_workspace_size(ctypes.byref(d), int(m), int(n), int(k)))


def save_size(s, n):
    return int(_lib.load().ns_save_size(int(s), int(n)))


def workspace(d, m, n, k=1, device="cuda"):
    nbytes = workspace_size(d, m, n, k)
    if nbytes == 0:
        raise NSError(_lib.NS_ERR_INVALID_ARG, "ns_workspace_size")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def ns_sketch(d, A, SA=None, ws=None, stream=None):
    """Algorithm 1 line 2: SA = S A (s x n, FP64, column-major)."""
    m, n = A.shape
    if SA is None:
        SA = _empty_cm(d.s, n, A.device)
    if ws is None:
        ws = workspace(d, m, n, 1, A.device)
    st = _lib.load().ns_sketch(ctypes.byref(d), _p(A), _dtype_code(A), m, n, _ld(A), _p(SA), _p(ws), ws.numel(),
                               _stream(stream))
    _lib.check(st, "ns_sketch")
    return SA


def sketch_rows_workspace(d, m_total, row_offset, m_p, n, device="cuda"):
    """Workspace tensor for ns_sketch_rows of rows [row_offset, row_offset + m_p)."""
    nbytes = int(_lib.load().ns_sketch_rows_workspace_size(ctypes.byref(d), int(m_total), int(row_offset),
                                                           int(m_p), int(n)))
    if nbytes == 0:
        raise NSError(_lib.NS_ERR_INVALID_ARG, "ns_sketch_rows_workspace_size")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def ns_sketch_rows(d, A_p, row_offset, m_total, SA=None, status=None, ws=None, stream=None):
    """The share S[:, o:o+m_p] A_p of the row block A_p = A[o:o+m_p, :] in the
    sketch of the whole m_total-row A (s x n FP64, column-major); the shares of
    blocks covering every row sum to ns_sketch's SA."""
    m_p, n = A_p.shape
    if SA is None:
        SA = _empty_cm(d.s, n, A_p.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A_p.device)
    lib = _lib.load()
    if ws is None:
        ws = sketch_rows_workspace(d, m_total, row_offset, m_p, n, A_p.device)
    st = lib.ns_sketch_rows(ctypes.byref(d), _p(A_p), _dtype_code(A_p), int(m_total), int(row_offset), m_p, n,
                            _ld(A_p), _p(SA), _p(status), _p(ws), ws.numel(), _stream(stream))
    _lib.check(st, "ns_sketch_rows")
    return SA


def ns_solve(d, A, k, save=True, status=None, ws=None, stream=None):
    """Algorithm 1: returns (Vk n x k, sigk k, save or None, status int32 tensor)."""
    m, n = A.shape
    dev = A.device
    Vk = _empty_cm(n, k, dev)
    sigk = torch.empty(k, dtype=torch.float64, device=dev)
    sv = None
    if save is True:
        sv = torch.empty(save_size(d.s, n), dtype=torch.float64, device=dev)
    elif isinstance(save, torch.Tensor):
        sv = save
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(d, m, n, k, dev)
    st = _lib.load().ns_solve(ctypes.byref(d), _p(A), _dtype_code(A), m, n, _ld(A), int(k), _p(Vk), _p(sigk),
                              _p(sv), _p(status), _p(ws), ws.numel(), _stream(stream))
    _lib.check(st, "ns_solve")
    return Vk, sigk, sv, status


def pipelined_workspace(d, m, n, device):
    nbytes = _lib.load().ns_solve_pipelined_workspace_size(ctypes.byref(d), m, n)
    if nbytes == 0:
        raise ValueError("invalid pipelined solve shape")
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def ns_solve_pipelined(d, As, k, status=None, ws=None, stream=None):
    """Algorithm 1 for the problems As (column-major device tensors of one shape and dtype), the
    sketch of problem i + 1 overlapping the dense stage of problem i: returns (Vk count x n x k as
    a list of n x k column-major views, sigk count x k, status int32 per problem)."""
    if not As:
        raise ValueError("no problems")
    m, n = As[0].shape
    dev = As[0].device
    for A in As:
        if A.shape != As[0].shape or A.dtype != As[0].dtype or _ld(A) != _ld(As[0]):
            raise ValueError("the problems must share shape, dtype and leading dimension")
    count = len(As)
    Vall = torch.empty(count * n * k, dtype=torch.float64, device=dev)
    sig = torch.empty(count * k, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.zeros(count, dtype=torch.int32, device=dev)
    if ws is None:
        ws = pipelined_workspace(d, m, n, dev)
    ptrs = (ctypes.c_void_p * count)(*[_p(A) for A in As])
    st = _lib.load().ns_solve_pipelined(ctypes.byref(d), ptrs, count, _dtype_code(As[0]), m, n, _ld(As[0]),
                                        int(k), _p(Vall), _p(sig), _p(status), _p(ws), ws.numel(),
                                        _stream(stream))
    _lib.check(st, "ns_solve_pipelined")
    Vks = [Vall[i * n * k:(i + 1) * n * k].view(k, n).t() for i in range(count)]
    return Vks, sig.view(count, k), status


def ns_solve_eps(d, A, eps, save=True, status=None, ws=None, stream=None):
    """Tolerance version of Algorithm 1: returns (Vk n x n, sigk n, k int32 tensor, save or None,
    status); columns 0..k-1 of Vk hold the right singular vectors with sigma < eps."""
    m, n = A.shape
    dev = A.device
    Vk = _empty_cm(n, n, dev)
    sigk = torch.empty(n, dtype=torch.float64, device=dev)
    kt = torch.zeros(1, dtype=torch.int32, device=dev)
    sv = None
    if save is True:
        sv = torch.empty(save_size(d.s, n), dtype=torch.float64, device=dev)
    elif isinstance(save, torch.Tensor):
        sv = save
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(d, m, n, 1, dev)
    st = _lib.load().ns_solve_eps(ctypes.byref(d), _p(A), _dtype_code(A), m, n, _ld(A), float(eps), _p(Vk),
                                  _p(sigk), _p(kt), _p(sv), _p(status), _p(ws), ws.numel(), _stream(stream))
    _lib.check(st, "ns_solve_eps")
    return Vk, sigk, kt, sv, status


def ns_sketch_update(d, m0, op, j, row, SA, stream=None):
    """Section 5 row update of a sketch in place: op NS_ROW_APPEND (row index j >= m0) or
    NS_ROW_REMOVE (row j); row is the row's n entries (device FP64), SA s x n column-major."""
    n = SA.shape[1]
    row = row.contiguous()
    st = _lib.load().ns_sketch_update(ctypes.byref(d), int(m0), int(op), int(j), _p(row), n, _p(SA),
                                      _stream(stream))
    _lib.check(st, "ns_sketch_update")
    return SA


def unpack_save(sv, s, n):
    """Views (SA s x n, V n x n, sigma n) of a save buffer."""
    SA = sv[: s * n].view(n, s).t()
    V = sv[s * n: s * n + n * n].view(n, n).t()
    sigma = sv[s * n + n * n: s * n + n * n + n]
    return SA, V, sigma


def ns_backward(d, m, n, k, save, Vk, dVk, dA=None, ws=None, stream=None):
    """Adjoint of ns_solve for a loss of W W^T: returns dL/dA (m x n, column-major)."""
    dev = save.device
    if dA is None:
        dA = _empty_cm(m, n, dev)
    if ws is None:
        ws = workspace(d, m, n, k, dev)
    st = _lib.load().ns_backward(ctypes.byref(d), int(m), int(n), int(k), _p(save), _p(Vk), _p(dVk), _p(dA),
                                 _ld(dA), _p(ws), ws.numel(), _stream(stream))
    _lib.check(st, "ns_backward")
    return dA


def ns_residual(A, W, ws=None, stream=None):
    """||A W||_F on the GPU (one FP64 pass over A); returns a 0-d device tensor."""
    m, n = A.shape
    out = torch.empty((), dtype=torch.float64, device=A.device)
    if ws is None:
        ws = torch.empty(8 * 4096, dtype=torch.uint8, device=A.device)
    st = _lib.load().ns_residual(_p(A), _dtype_code(A), m, n, _ld(A), _p(W), W.shape[1], _p(out), _p(ws),
                                 ws.numel(), _stream(stream))
    _lib.check(st, "ns_residual")
    return out


def ns_srht_meta(d, m, stream=None, device="cuda"):
    """(sign_words uint32 as int32 tensor, rows int32) of the SRHT realisation."""
    lg = max(int(m - 1).bit_length(), 0)
    nwords = ((1 << lg) + 31) // 32
    words = torch.empty(nwords, dtype=torch.int32, device=device)
    rows = torch.empty(d.s, dtype=torch.int32, device=device)
    st = _lib.load().ns_srht_meta(ctypes.byref(d), int(m), _p(words), _p(rows), _stream(stream))
    _lib.check(st, "ns_srht_meta")
    return words, rows


def ns_sparse_meta(d, m, stream=None, device="cuda"):
    """(rows m x zeta int32, signs m x zeta int8) of the sparse-sign realisation."""
    rows = torch.empty((m, d.zeta), dtype=torch.int32, device=device)
    signs = torch.empty((m, d.zeta), dtype=torch.int8, device=device)
    st = _lib.load().ns_sparse_meta(ctypes.byref(d), int(m), _p(rows), _p(signs), _stream(stream))
    _lib.check(st, "ns_sparse_meta")
    return rows, signs


def ns_sketch_static(d, A, SA=None, status=None, stream=None):
    """SRHT sketch using the library's own fixed scratch array: no workspace is
    passed and nothing is allocated by the call (the output SA and the status
    word are allocated here only if the caller did not pass them)."""
    m, n = A.shape
    if SA is None:
        SA = _empty_cm(d.s, n, A.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = _lib.load().ns_sketch_static(ctypes.byref(d), _p(A), _dtype_code(A), m, n, _ld(A), _p(SA), _p(status),
                                      _stream(stream))
    _lib.check(st, "ns_sketch_static")
    return SA, status


def ns_solve_batched(problems, stream=None, ws=None, device="cuda", tuning=None):
    """Batched Algorithm 1.  problems: list of dicts with A (column-major CUDA
    tensor, float64 or float32: the FP32-stream sketch), s, k, seed and
    optionally tls=True.  tuning: None (keep the current launch geometry) or a
    dict with panel, sketch_ctas_per_sm, dense_ctas_per_sm (see
    paper_2206_00975_gb300.autotune; the results do not depend on it).
    Returns (list of (Vk, sigk, x), status int32 tensor, keep-alive tuple)."""
    n_b = len(problems)
    arr = (Problem * n_b)()
    outs = []
    any32 = False
    for i, p in enumerate(problems):
        A = p["A"]
        m, n = A.shape
        k = int(p.get("k", 1))
        Vk = _empty_cm(n, k, A.device)
        sigk = torch.empty(k, dtype=torch.float64, device=A.device)
        x = torch.empty(max(n - 1, 1), dtype=torch.float64, device=A.device) if p.get("tls") else None
        outs.append((Vk, sigk, x))
        dt = _dtype_code(A)
        any32 = any32 or dt == NS_F32
        arr[i] = Problem(A.data_ptr(), m, n, _ld(A), int(p["s"]), k, 1 if p.get("tls") else 0,
                         int(p.get("seed", 0)) & ((1 << 64) - 1), Vk.data_ptr(), sigk.data_ptr(),
                         x.data_ptr() if x is not None else 0, dt, 0)
    raw = bytes(arr)
    dev_arr = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
    status = torch.zeros(n_b, dtype=torch.int32, device=device)
    d = desc(NS_SRHT, s=1, seed=0, prec=NS_PREC_FP32_STREAM if any32 else NS_PREC_FP64)
    lib = _lib.load()
    if tuning is not None:
        _lib.check(lib.ns_batched_tuning(int(tuning.get("panel", 0)), int(tuning.get("sketch_ctas_per_sm", 0)),
                                         int(tuning.get("dense_ctas_per_sm", 0))), "ns_batched_tuning")
    nbytes = int(lib.ns_batched_workspace_size(ctypes.byref(d), n_b, ctypes.byref(arr)))
    if nbytes == 0:
        raise NSError(_lib.NS_ERR_INVALID_ARG, "ns_batched_workspace_size")
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    st = lib.ns_solve_batched(ctypes.byref(d), n_b, ctypes.byref(arr), _p(dev_arr), _p(status), _p(ws), ws.numel(),
                              _stream(stream))
    _lib.check(st, "ns_solve_batched")
    # keep the device copy of the descriptors alive until the work is done
    outs_ref = (outs, dev_arr, ws)
    return outs_ref[0], status, outs_ref


def batched_supports_fp32():
    """ns_problem carries a dtype: FP32 problems take the FP32-stream sketch."""
    return True


def ns_aaa_real(x, f, K, smax, seed=0, forced=None, want_sketch=False, ws=None, stream=None):
    """AAA with a reused SRHT sketch (Section 6.2) on the GPU.  x, f: CUDA float64
    vectors.  Returns dict(support, W, errmax, status[, SAk]) as device tensors."""
    m = x.numel()
    dev = x.device
    d = desc(NS_SRHT, s=smax, seed=seed)
    lib = _lib.load()
    nbytes = int(lib.ns_aaa_workspace_size(ctypes.byref(d), m, int(K)))
    if nbytes == 0:
        raise NSError(_lib.NS_ERR_INVALID_ARG, "ns_aaa_workspace_size")
    if ws is None:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {"support": torch.empty(K, dtype=torch.int64, device=dev),
           "W": torch.empty((K, K), dtype=torch.float64, device=dev),
           "errmax": torch.empty(K, dtype=torch.float64, device=dev),
           "status": torch.zeros(1, dtype=torch.int32, device=dev)}
    SAk = _empty_cm(smax, K, dev) if want_sketch else None
    st = lib.ns_aaa_real(ctypes.byref(d), _p(x), _p(f), m, int(K), _p(forced), _p(out["support"]), _p(out["W"]),
                         _p(out["errmax"]), _p(SAk), _p(out["status"]), _p(ws), ws.numel(), _stream(stream))
    _lib.check(st, "ns_aaa_real")
    if want_sketch:
        out["SAk"] = SAk
    out["_ws"] = ws
    return out


def ns_solve_sketched(d, SA, k, save=False, status=None, ws=None, stream=None):
    """Lines 3-4 of Algorithm 1 on a given sketch SA (s x n, column-major)."""
    s_, n = SA.shape
    dev = SA.device
    Vk = _empty_cm(n, k, dev)
    sigk = torch.empty(k, dtype=torch.float64, device=dev)
    sv = torch.empty(save_size(d.s, n), dtype=torch.float64, device=dev) if save is True else (
        save if isinstance(save, torch.Tensor) else None)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=dev)
    if ws is None:
        ws = workspace(d, max(n, d.s), n, k, dev)
    st = _lib.load().ns_solve_sketched(ctypes.byref(d), _p(SA), n, int(k), _p(Vk), _p(sigk), _p(sv), _p(status),
                                       _p(ws), ws.numel(), _stream(stream))
    _lib.check(st, "ns_solve_sketched")
    return Vk, sigk, sv, status


def jacobi_stats(d, m, n, ws, sketched=False, stream=None):
    """(FP64 full sweeps, FP64 rotations, check passes, ring cluster size or 0, FP32-phase sweeps,
    FP32-phase rotations, completions with K^4 and K^6 terms, 1 if the convergence test ran on the
    Gram matrix after the completions) of the last solve in workspace ws."""
    out = torch.zeros(8, dtype=torch.int64, device=ws.device)
    lib = _lib.load()
    if sketched:
        st = lib.ns_sketched_stats(ctypes.byref(d), int(n), _p(ws), _p(out), _stream(stream))
    else:
        st = lib.ns_solve_stats(ctypes.byref(d), int(m), int(n), _p(ws), _p(out), _stream(stream))
    _lib.check(st, "jacobi_stats")
    return [int(v) for v in out.cpu()]
