"""ctypes loader for libns.so (the C ABI declared in include/ns.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libns.  There is no CPU fallback: if the library is missing the
first call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libns.so")

NS_OK, NS_ERR_INVALID_ARG, NS_ERR_WORKSPACE, NS_ERR_NONFINITE = 0, 1, 2, 3
NS_ERR_NOCONV, NS_ERR_TLS_NOSOLUTION, NS_ERR_TIMEOUT, NS_ERR_CUDA = 4, 5, 6, 7
NS_SRHT, NS_SPARSE_SIGN, NS_GAUSSIAN, NS_HRHT = 0, 1, 2, 3
NS_F64, NS_F32 = 0, 1
NS_PREC_FP64, NS_PREC_FP32_STREAM, NS_PREC_BF16X3 = 0, 1, 2
NS_ROW_APPEND, NS_ROW_REMOVE = 0, 1

# every symbol include/ns.h declares
EXPORTS = [
    "ns_status_string", "ns_version", "ns_workspace_size", "ns_save_size", "ns_sketch", "ns_solve",
    "ns_backward", "ns_residual", "ns_srht_meta", "ns_sparse_meta", "ns_sketch_static",
    "ns_batched_workspace_size", "ns_solve_batched", "ns_aaa_workspace_size", "ns_aaa_real",
    "ns_solve_sketched", "ns_solve_stats", "ns_sketched_stats", "ns_solve_eps", "ns_sketch_update",
    "ns_test_bounded_wait", "ns_batched_tuning", "ns_sketch_rows", "ns_sketch_rows_workspace_size",
    "ns_solve_pipelined", "ns_solve_pipelined_workspace_size",
]


class SketchDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("zeta", ctypes.c_int32), ("s", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int32), ("max_sweeps", ctypes.c_int32)]


class Problem(ctypes.Structure):
    """ns_problem of include/ns.h (device pointers inside)."""
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("s", ctypes.c_int64), ("k", ctypes.c_int32), ("tls", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("Vk", ctypes.c_void_p), ("sigk", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class NSError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s" % (what, status_string(status)))


_lib = None


def load():
    """Load libns.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libns.so not found at %s; build it with python -m paper_2206_00975_gb300.build"
                           % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    D = ctypes.POINTER(SketchDesc)
    sig = {
        "ns_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "ns_version": (ctypes.c_char_p, []),
        "ns_workspace_size": (sz, [D, i64, i64, i32]),
        "ns_save_size": (i64, [i64, i64]),
        "ns_sketch": (ctypes.c_int, [D, P, i32, i64, i64, i64, P, P, sz, P]),
        "ns_solve": (ctypes.c_int, [D, P, i32, i64, i64, i64, i32, P, P, P, P, P, sz, P]),
        "ns_backward": (ctypes.c_int, [D, i64, i64, i32, P, P, P, P, i64, P, sz, P]),
        "ns_residual": (ctypes.c_int, [P, i32, i64, i64, i64, P, i32, P, P, sz, P]),
        "ns_srht_meta": (ctypes.c_int, [D, i64, P, P, P]),
        "ns_sparse_meta": (ctypes.c_int, [D, i64, P, P, P]),
        "ns_sketch_static": (ctypes.c_int, [D, P, i32, i64, i64, i64, P, P, P]),
        "ns_batched_workspace_size": (sz, [D, i32, P]),
        "ns_solve_batched": (ctypes.c_int, [D, i32, P, P, P, P, sz, P]),
        "ns_aaa_workspace_size": (sz, [D, i64, i32]),
        "ns_aaa_real": (ctypes.c_int, [D, P, P, i64, i32, P, P, P, P, P, P, P, sz, P]),
        "ns_solve_sketched": (ctypes.c_int, [D, P, i64, i32, P, P, P, P, P, sz, P]),
        "ns_solve_stats": (ctypes.c_int, [D, i64, i64, P, P, P]),
        "ns_sketched_stats": (ctypes.c_int, [D, i64, P, P, P]),
        "ns_solve_eps": (ctypes.c_int, [D, P, i32, i64, i64, i64, ctypes.c_double, P, P, P, P, P, P, sz, P]),
        "ns_sketch_update": (ctypes.c_int, [D, i64, i32, i64, P, i64, P, P]),
        "ns_test_bounded_wait": (ctypes.c_int, [i32, i64, P, P, sz, P]),
        "ns_batched_tuning": (ctypes.c_int, [i32, i32, i32]),
        "ns_sketch_rows_workspace_size": (sz, [D, i64, i64, i64, i64]),
        "ns_solve_pipelined_workspace_size": (sz, [D, i64, i64]),
        "ns_solve_pipelined": (ctypes.c_int, [D, P, i32, i32, i64, i64, i64, i32, P, P, P, P, sz, P]),
        "ns_sketch_rows": (ctypes.c_int, [D, P, i32, i64, i64, i64, i64, i64, P, P, P, sz, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status):
    try:
        return load().ns_status_string(int(status)).decode()
    except Exception:  # pragma: no cover - only when the library itself is missing
        return "status %d" % int(status)


def check(status, what):
    if status != NS_OK:
        raise NSError(status, what)
