"""Seeded synthetic inputs for the null-space workloads.

This module only builds test matrices from numpy's ``default_rng``; it holds
none of the sketch-and-solve arithmetic.  Both the GPU tests and the oracle
tests (and the benchmark) consume the exact bytes produced here, so the two
sides always see identical inputs.

Shapes and spectra follow the workloads measured by the benchmark:

* plain FP64:   m=4096, n=32, A = U diag(sigma) V^T, sigma_1..31 log-spaced
  from 1 to 1e-4, sigma_32 = 1e-12 (k = 1, SRHT s = 128);
* at scale:     m=2^20, n=256, sigma_1..252 log-spaced from 1 to 1e-6 and an
  exact null space of dimension 4 (k = 4, s = 1024);
* precision:    m=2^22, n=512, sigma graded from 1 to 1e-6, trailing two 1e-9,
  stored FP32 (k = 2, s = 2048);
* adjoint:      m=2^18, n=128, 120 singular values of a Gaussian plus eight in
  [1e-8, 1e-6] (k = 8, s = 512);
* batched TLS:  [X b] with X Gaussian, b = X x_true + 1e-3 noise;
* AAA:          sorted uniform points in [-1, 1], f = tanh(50 x).

U is the Q factor of a seeded Gaussian (numpy/LAPACK QR), V likewise.  All
matrices are returned column-major (Fortran order).
"""
import numpy as np


def orthonormal(rng, m, n):
    """Q factor (m x n, orthonormal columns) of an m x n standard Gaussian."""
    q, r = np.linalg.qr(rng.standard_normal((m, n)))
    return np.asfortranarray(q * np.sign(np.diag(r)))


def from_svd(U, sigma, V):
    return np.asfortranarray((U * sigma) @ V.T)


def plain(seed=0, m=4096, n=32):
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, m, n)
    V = orthonormal(rng, n, n)
    sigma = np.concatenate([np.logspace(0, -4, n - 1), [1e-12]])
    return {"A": from_svd(U, sigma, V), "U": U, "sigma": sigma, "V": V, "k": 1, "s": 4 * n}


def at_scale(seed=0, m=1 << 20, n=256, null_dim=4):
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, m, n)
    V = orthonormal(rng, n, n)
    sigma = np.concatenate([np.logspace(0, -6, n - null_dim), np.zeros(null_dim)])
    return {"A": from_svd(U, sigma, V), "U": U, "sigma": sigma, "V": V, "k": null_dim, "s": 4 * n}


def graded(seed=0, m=1 << 12, n=64, k=2, tail=1e-9, dtype=np.float64):
    """Precision workload: sigma log-spaced 1..1e-6 with k trailing values `tail`."""
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, m, n)
    V = orthonormal(rng, n, n)
    sigma = np.concatenate([np.logspace(0, -6, n - k), np.full(k, tail)])
    A = from_svd(U, sigma, V).astype(dtype)
    return {"A": np.asfortranarray(A), "U": U, "sigma": sigma, "V": V, "k": k, "s": 4 * n}


def adjoint(seed=0, m=1 << 18, n=128, rank=120, k=8):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, rank))
    top = np.linalg.svd(G, compute_uv=False)
    sigma = np.concatenate([top, np.logspace(-6, -8, n - rank)])
    U = orthonormal(rng, m, n)
    V = orthonormal(rng, n, n)
    W = np.random.default_rng(seed + 1).standard_normal((n, 16))
    return {"A": from_svd(U, sigma, V), "U": U, "sigma": sigma, "V": V, "k": k, "s": 4 * n,
            "W": np.asfortranarray(W)}


def tls_problem(rng, m, n, noise=1e-3):
    X = rng.standard_normal((m, n))
    x_true = rng.standard_normal(n)
    b = X @ x_true + noise * rng.standard_normal(m)
    return np.asfortranarray(np.column_stack([X, b])), x_true


def tls_batch_shapes(seed, batch, m_lo=1 << 11, m_hi=1 << 16, n_lo=8, n_hi=128):
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=batch)
    ns = rng.integers(n_lo, n_hi + 1, size=batch)
    return ms.astype(np.int64), ns.astype(np.int64)


def aaa_points(seed=0, m=1 << 17, scale=50.0):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(-1.0, 1.0, size=m))
    # strictly increasing (duplicates would make the Loewner matrix undefined)
    x = np.unique(x)
    while x.size < m:
        x = np.unique(np.concatenate([x, rng.uniform(-1.0, 1.0, size=m - x.size)]))
    return x, np.tanh(scale * x)
