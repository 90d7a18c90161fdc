"""Oracle: plain, slow FP64 CPU reference of the sketch-and-solve null-space method
(Park & Nakatsukasa, "A Fast Randomized Algorithm for Computing an Approximate
Null Space", Algorithm 1 and Sections 4-6).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library never
imports it and shares no code with it.  The arithmetic lives in ``oracle.c``;
this module only builds it with gcc and marshals numpy arrays through ctypes.

Every function names the passage of the paper it follows.  Matrices are
column-major (Fortran order) float64 unless stated otherwise.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None

OK, ERR_INVALID_ARG, ERR_NOCONV, ERR_TLS_NOSOLUTION = 0, 1, 4, 5
SRHT, SPARSE_SIGN, GAUSSIAN, HRHT = 0, 1, 2, 3


def build(force=False):
    """Compile oracle.c into _oracle.so with gcc (plain -O2, no tuning)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, i32, u64, dbl, i = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        sig = {
            "or_philox4x64_10": (None, [P, P, P]),
            "or_ceil_log2": (i, [i64]),
            "or_signs": (None, [u64, i64, P]),
            "or_prp": (i64, [u64, i, i64]),
            "or_sample_rows": (None, [u64, i, i64, P]),
            "or_fwht": (None, [P, i64]),
            "or_srht": (i, [u64, i64, P, i64, i64, i64, i, P]),
            "or_srht_explicit": (i, [u64, i64, i64, P]),
            "or_hash_rows": (None, [u64, i64, i64, P, P]),
            "or_hrht": (i, [u64, i64, P, i64, i64, i64, i, P]),
            "or_hrht_explicit": (i, [u64, i64, i64, P]),
            "or_sparse_sign_cols": (None, [u64, i64, i32, i64, P, P]),
            "or_sparse_sign": (i, [u64, i64, i32, P, i64, i64, i64, i, P]),
            "or_gaussian_entry": (dbl, [u64, i64, i64]),
            "or_gaussian": (i, [u64, i64, P, i64, i64, i64, P, i64, P]),
            "or_gaussian_rows": (i, [u64, i64, P, i64, i64, i64, P, i64, P, P]),
            "or_householder_qr": (i, [P, i64, i64, i64, P]),
            "or_jacobi": (i, [P, i64, P, P, dbl, i, P]),
            "or_extract": (None, [P, P, i64, i32, P, P, P]),
            "or_count_below": (ctypes.c_int32, [P, i64, ctypes.c_double]),
            "or_sketch_update": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, i64, i32, i64, ctypes.c_int, i64, P,
                                                i64, P]),
            "or_sketch": (i, [i, u64, i64, i32, P, i64, i64, i64, P]),
            "or_solve_sketched": (i, [P, i64, i64, i32, P, P, P, P, P]),
            "or_solve": (i, [i, u64, i64, i32, P, i64, i64, i64, i32, P, P, P, P, P]),
            "or_residual": (dbl, [P, i64, i64, i64, P, i32]),
            "or_tls": (i, [u64, i64, P, i64, i64, i64, P, P]),
            "or_backward_srht": (i, [u64, i64, i64, i64, i32, P, P, P, P, P, P, i64]),
            "or_aaa": (i, [u64, P, P, i64, i32, i64, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    return np.asfortranarray(a, dtype=np.float64)


def _check(st, what):
    if st not in (OK, ERR_NOCONV):
        raise ValueError("oracle %s failed with status %d" % (what, st))
    return st


# ----------------------------------------------------------------------------
# Random streams (Philox4x64-10, Salmon et al. SC'11)
# ----------------------------------------------------------------------------
def philox4x64_10(ctr, key):
    """One Philox4x64-10 block: 4 uint64 words for counter ctr[4], key key[2]."""
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().or_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def ceil_log2(m):
    return int(_load().or_ceil_log2(int(m)))


def signs(seed, length):
    """Diagonal of D in the SRFT (Section 2): int8 array of +-1."""
    d = np.zeros(int(length), dtype=np.int8)
    _load().or_signs(ctypes.c_uint64(seed), int(length), _p(d))
    return d


def prp(seed, lg, x):
    return int(_load().or_prp(ctypes.c_uint64(seed), int(lg), int(x)))


def sample_rows(seed, lg, s):
    """Coordinates kept by R in the SRFT (Section 2), in draw order."""
    r = np.zeros(int(s), dtype=np.int64)
    _load().or_sample_rows(ctypes.c_uint64(seed), int(lg), int(s), _p(r))
    return r


def fwht(x):
    """Sylvester-ordered unnormalised Walsh-Hadamard transform (recursive)."""
    y = np.array(x, dtype=np.float64).copy()
    assert y.ndim == 1 and (y.size & (y.size - 1)) == 0
    _load().or_fwht(_p(y), y.size)
    return y


# ----------------------------------------------------------------------------
# Sketches (Algorithm 1 line 2)
# ----------------------------------------------------------------------------
def srht(seed, s, A, scaled=True):
    """SA = (1/sqrt s) R H D [A; 0] (the SRFT of Section 2 with H for F)."""
    A = _f64(A)
    m, n = A.shape
    SA = np.zeros((s, n), dtype=np.float64, order="F")
    _check(_load().or_srht(ctypes.c_uint64(seed), s, _p(A), m, n, max(m, 1), int(scaled), _p(SA)), "srht")
    return SA


def srht_explicit(seed, s, m):
    """Explicit unscaled SRHT matrix S[t, j] = d_j (-1)^popcount(r_t & j), s x m."""
    S = np.zeros((s, m), dtype=np.float64, order="F")
    _check(_load().or_srht_explicit(ctypes.c_uint64(seed), s, m, _p(S)), "srht_explicit")
    return S


def hash_rows(seed, s, mp):
    """The 1-hashing matrix of the H-RHT (Section 2): row h[i] (int64) and sign
    sg[i] (int8) of coordinate i < mp."""
    h = np.zeros(int(mp), dtype=np.int64)
    sg = np.zeros(int(mp), dtype=np.int8)
    _load().or_hash_rows(ctypes.c_uint64(seed), int(s), int(mp), _p(h), _p(sg))
    return h, sg


def hrht(seed, s, A, scaled=True):
    """SA = S_h (1/sqrt m') H D [A; 0], the H-RHT of Section 2."""
    A = _f64(A)
    m, n = A.shape
    SA = np.zeros((s, n), dtype=np.float64, order="F")
    _check(_load().or_hrht(ctypes.c_uint64(seed), s, _p(A), m, n, max(m, 1), int(scaled), _p(SA)), "hrht")
    return SA


def hrht_explicit(seed, s, m):
    """Explicit unscaled H-RHT matrix, s x m: S[t, j] = d_j sum_{h[i]=t} sg[i] (-1)^popcount(i & j)."""
    S = np.zeros((s, m), dtype=np.float64, order="F")
    _check(_load().or_hrht_explicit(ctypes.c_uint64(seed), s, m, _p(S)), "hrht_explicit")
    return S


def sparse_sign_cols(seed, s, zeta, m):
    """Rows (m x zeta int32) and signs (m x zeta int8) of the sparse-sign sketch columns."""
    rows = np.zeros((m, zeta), dtype=np.int32)
    sg = np.zeros((m, zeta), dtype=np.int8)
    _load().or_sparse_sign_cols(ctypes.c_uint64(seed), s, zeta, m, _p(rows), _p(sg))
    return rows, sg


def sparse_sign(seed, s, zeta, A, scaled=True):
    A = _f64(A)
    m, n = A.shape
    SA = np.zeros((s, n), dtype=np.float64, order="F")
    _check(_load().or_sparse_sign(ctypes.c_uint64(seed), s, zeta, _p(A), m, n, max(m, 1), int(scaled), _p(SA)),
           "sparse_sign")
    return SA


def gaussian_entry(seed, r, j):
    return float(_load().or_gaussian_entry(ctypes.c_uint64(seed), int(r), int(j)))


def gaussian(seed, s, A, cols=None):
    """SA = G A / sqrt(s) (Theorem 2.1 scaling); only columns `cols` are formed if given."""
    A = _f64(A)
    m, n = A.shape
    SA = np.zeros((s, n), dtype=np.float64, order="F")
    if cols is None:
        _check(_load().or_gaussian(ctypes.c_uint64(seed), s, _p(A), m, n, max(m, 1), None, n, _p(SA)), "gaussian")
    else:
        c = np.ascontiguousarray(cols, dtype=np.int64)
        _check(_load().or_gaussian(ctypes.c_uint64(seed), s, _p(A), m, n, max(m, 1), _p(c), c.size, _p(SA)),
               "gaussian")
    return SA


def gaussian_rows(seed, s, A, rows):
    """Rows `rows` of SA = G A / sqrt(s) (every column), and the size of their
    terms sqrt(sum_j (G(r, j) A(j, c))^2) / sqrt(s): returns (out, mag), both
    len(rows) x n."""
    A = _f64(A)
    m, n = A.shape
    r = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros((r.size, n), dtype=np.float64, order="F")
    mag = np.zeros((r.size, n), dtype=np.float64, order="F")
    _check(_load().or_gaussian_rows(ctypes.c_uint64(seed), s, _p(A), m, n, max(m, 1), _p(r), r.size, _p(out),
                                    _p(mag)), "gaussian_rows")
    return out, mag


def sketch(kind, seed, s, A, zeta=8):
    A = _f64(A)
    m, n = A.shape
    SA = np.zeros((s, n), dtype=np.float64, order="F")
    _check(_load().or_sketch(int(kind), ctypes.c_uint64(seed), s, zeta, _p(A), m, n, max(m, 1), _p(SA)), "sketch")
    return SA


# ----------------------------------------------------------------------------
# Dense part (Algorithm 1 lines 3-4)
# ----------------------------------------------------------------------------
def householder_qr_r(B):
    """R factor (n x n) of the Householder QR of B (s x n)."""
    B = _f64(B)
    s, n = B.shape
    R = np.zeros((n, n), dtype=np.float64, order="F")
    _check(_load().or_householder_qr(_p(B), s, n, s, _p(R)), "householder_qr")
    return R


def jacobi(X, tol=None, max_sweeps=30):
    """One-sided Jacobi SVD of square X: returns (X V, V, sigma, sweeps, status)."""
    X = _f64(X).copy(order="F")
    n = X.shape[0]
    assert X.shape == (n, n)
    V = np.zeros((n, n), dtype=np.float64, order="F")
    sig = np.zeros(n, dtype=np.float64)
    sw = ctypes.c_int(0)
    if tol is None:
        tol = n * 2.0 ** -53
    st = _load().or_jacobi(_p(X), n, _p(V), _p(sig), float(tol), int(max_sweeps), ctypes.byref(sw))
    return X, V, sig, sw.value, st


def extract(sigma, V, k):
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    V = _f64(V)
    n = V.shape[0]
    Vk = np.zeros((n, k), dtype=np.float64, order="F")
    sk = np.zeros(k, dtype=np.float64)
    order = np.zeros(n, dtype=np.int64)
    _load().or_extract(_p(sigma), _p(V), n, k, _p(Vk), _p(sk), _p(order))
    return Vk, sk, order


def solve_sketched(SA, k):
    """Lines 3-4 of Algorithm 1 on a formed sketch: (Vk, sigk, V_full, sigma_full, sweeps, status)."""
    SA = _f64(SA)
    s, n = SA.shape
    Vk = np.zeros((n, k), dtype=np.float64, order="F")
    sk = np.zeros(k, dtype=np.float64)
    V = np.zeros((n, n), dtype=np.float64, order="F")
    sig = np.zeros(n, dtype=np.float64)
    sw = ctypes.c_int(0)
    st = _check(_load().or_solve_sketched(_p(SA), s, n, k, _p(Vk), _p(sk), _p(V), _p(sig), ctypes.byref(sw)),
                "solve_sketched")
    return Vk, sk, V, sig, sw.value, st


def solve(kind, seed, s, A, k, zeta=8):
    """Algorithm 1 end to end: dict with Vk, sigk, SA, V, sigma, status."""
    A = _f64(A)
    m, n = A.shape
    Vk = np.zeros((n, k), dtype=np.float64, order="F")
    sk = np.zeros(k, dtype=np.float64)
    SA = np.zeros((s, n), dtype=np.float64, order="F")
    V = np.zeros((n, n), dtype=np.float64, order="F")
    sig = np.zeros(n, dtype=np.float64)
    st = _check(_load().or_solve(int(kind), ctypes.c_uint64(seed), s, zeta, _p(A), m, n, max(m, 1), k, _p(Vk),
                                 _p(sk), _p(SA), _p(V), _p(sig)), "solve")
    return {"Vk": Vk, "sigk": sk, "SA": SA, "V": V, "sigma": sig, "status": st}


def solve_eps(kind, seed, s, A, eps, zeta=8):
    """The tolerance version of Algorithm 1 (Section 2, after Algorithm 1): every right
    singular vector of SA with sigma < eps.  Returns (Vk n x k, sigk k, k, full solve dict)."""
    A = _f64(A)
    n = A.shape[1]
    full = solve(kind, seed, s, A, 1, zeta=zeta)
    sig = np.ascontiguousarray(full["sigma"], dtype=np.float64)
    k = int(_load().or_count_below(_p(sig), n, float(eps)))
    if k == 0:
        return np.zeros((n, 0), order="F"), np.zeros(0), 0, full
    Vk, sk, _ = extract(sig, full["V"], k)
    return Vk, sk, k, full


def sketch_update(kind, seed, s, SA, m0, op, j, row, zeta=8):
    """Section 5 row update of a sketch (op 0: Algorithm 2, append row j >= m0; op 1:
    Algorithm 3, remove row j).  Returns the updated copy of SA."""
    SA = _f64(SA).copy(order="F")
    row = np.ascontiguousarray(row, dtype=np.float64)
    _check(_load().or_sketch_update(int(kind), ctypes.c_uint64(seed), int(s), int(zeta), int(m0), int(op), int(j),
                                    _p(row), row.size, _p(SA)), "sketch_update")
    return SA


def residual(A, W):
    """||A W||_F (the objective of Problem 2.1)."""
    A = _f64(A)
    W = _f64(W)
    m, n = A.shape
    return float(_load().or_residual(_p(A), m, n, max(m, 1), _p(W), W.shape[1]))


def tls(seed, s, Xb):
    """Sketched TLS (Section 4): returns (x, v, status)."""
    Xb = _f64(Xb)
    m, n1 = Xb.shape
    x = np.zeros(n1 - 1, dtype=np.float64)
    v = np.zeros(n1, dtype=np.float64)
    st = _load().or_tls(ctypes.c_uint64(seed), s, _p(Xb), m, n1, m, _p(x), _p(v))
    if st not in (OK, ERR_NOCONV, ERR_TLS_NOSOLUTION):
        raise ValueError("oracle tls failed with status %d" % st)
    return x, v, st


def backward_srht(seed, s, m, SA, V, sigma, Vk, dVk):
    """dL/dA for a loss of W W^T, through the SVD of SA and S^T (SRHT)."""
    SA, V, Vk, dVk = _f64(SA), _f64(V), _f64(Vk), _f64(dVk)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    n = V.shape[0]
    k = Vk.shape[1]
    dA = np.zeros((m, n), dtype=np.float64, order="F")
    _check(_load().or_backward_srht(ctypes.c_uint64(seed), s, m, n, k, _p(SA), _p(V), _p(sigma), _p(Vk), _p(dVk),
                                    _p(dA), m), "backward_srht")
    return dA


def aaa(seed, x, f, K, smax, forced=None, return_sketch=False):
    """Sketched AAA with sketch reuse (Section 6.2): (support, W, errmax, status[, SAk])."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    m = x.size
    sup = np.zeros(K, dtype=np.int64)
    W = np.zeros((K, K), dtype=np.float64)
    err = np.zeros(K, dtype=np.float64)
    fp = None if forced is None else np.ascontiguousarray(forced, dtype=np.int64)
    SAk = np.zeros((smax, K), dtype=np.float64, order="F")
    st = _check(_load().or_aaa(ctypes.c_uint64(seed), _p(x), _p(f), m, K, smax, _p(fp), _p(sup), _p(W), _p(err),
                               _p(SAk)), "aaa")
    if return_sketch:
        return sup, W, err, st, SAk
    return sup, W, err, st
