"""Pins of the oracle to things other than itself.

Each test checks one oracle routine against a third-party implementation used
as a black box (numpy's Philox, scipy's Hadamard matrix, LAPACK QR/SVD, torch
autograd), an exact identity the paper states, a deterministic bound of the
paper evaluated on the realized sketch, or brute force on tiny inputs.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle as O
from paper_2206_00975_gb300 import workloads
from tests.helpers import chi, orth, sine

U53 = 2.0 ** -53


# ---------------------------------------------------------------- Philox ----
@pytest.mark.parametrize("ctr,key", [
    ([1, 0, 0, 0], [0, 0]),
    ([5, 7, 1, 0], [123, 0]),
    ([2 ** 40 + 3, 2 ** 63 + 11, 3, 0], [0xDEADBEEFCAFEF00D, 0]),
    ([9, 1, 2, 77], [42, 0x1234567890ABCDEF]),
])
def test_philox_matches_numpy(ctr, key):
    # numpy.random.Philox(counter=c) emits the block of counter c+1 first.
    prev = list(ctr)
    prev[0] -= 1
    # pass uint64 arrays: numpy converts plain ints >= 2^63 through float64
    raw = np.random.Philox(counter=np.array(prev, dtype=np.uint64),
                           key=np.array(key, dtype=np.uint64)).random_raw(4)
    assert np.array_equal(raw, O.philox4x64_10(ctr, key))


# ------------------------------------------------------------------ FWHT ----
@pytest.mark.parametrize("lg", [0, 1, 3, 6])
def test_fwht_equals_scipy_hadamard(lg):
    n = 1 << lg
    H = scipy.linalg.hadamard(n).astype(np.float64)       # Sylvester order
    cols = np.column_stack([O.fwht(np.eye(n)[:, j]) for j in range(n)])
    assert np.array_equal(cols, H)
    assert np.array_equal(cols @ cols.T, n * np.eye(n))   # H H^T = m' I


def test_fwht_twice_is_scaled_identity_on_integers():
    rng = np.random.default_rng(1)
    x = rng.integers(-1000, 1000, size=1 << 12).astype(np.float64)
    assert np.array_equal(O.fwht(O.fwht(x)), (1 << 12) * x)


def test_fwht_popcount_form():
    n = 64
    i = np.arange(n)
    for j in (0, 1, 5, 33, 63):
        e = np.zeros(n)
        e[j] = 1.0
        expect = np.where([bin(v & j).count("1") % 2 for v in i], -1.0, 1.0)
        assert np.array_equal(O.fwht(e), expect)


# ---------------------------------------------------- SRFT ingredients ----
def test_signs_balanced_and_seeded():
    d = O.signs(5, 1 << 16)
    assert set(np.unique(d)) == {-1, 1}
    assert abs(d.astype(np.int64).sum()) < 5 * np.sqrt(1 << 16)
    assert not np.array_equal(d, O.signs(6, 1 << 16))
    assert np.array_equal(d[:1000], O.signs(5, 1000))    # prefix-stable


@pytest.mark.parametrize("lg", [1, 2, 5, 10, 13])
def test_sample_rows_is_permutation(lg):
    r = O.sample_rows(11, lg, 1 << lg)
    assert np.array_equal(np.sort(r), np.arange(1 << lg))


def test_sample_rows_prefix_uniform():
    # first draw over many seeds must be uniform on [0, m')  (chi-square)
    lg = 6
    first = np.array([O.prp(seed, lg, 0) for seed in range(6400)])
    counts = np.bincount(first, minlength=1 << lg)
    p = scipy.stats.chisquare(counts).pvalue
    assert p > 1e-4
    # pairs (r_0, r_1) are distinct and r_1 is uniform on the remaining values
    second = np.array([O.prp(seed, lg, 1) for seed in range(6400)])
    assert np.all(first != second)


def test_srht_explicit_equals_hadamard_construction():
    # S = R H D built from scipy's Hadamard matrix, the signs and the rows
    seed, m, s = 9, 45, 20
    lg = O.ceil_log2(m)
    H = scipy.linalg.hadamard(1 << lg).astype(np.float64)
    D = np.diag(O.signs(seed, 1 << lg).astype(np.float64))
    rows = O.sample_rows(seed, lg, s)
    S_ref = (H @ D)[rows, :m]
    assert np.array_equal(O.srht_explicit(seed, s, m), S_ref)


@pytest.mark.parametrize("m,n,s", [(64, 7, 32), (37, 5, 16), (1, 1, 1), (2, 2, 2), (33, 3, 64)])
def test_srht_matches_explicit_S_bitexact(m, n, s):
    rng = np.random.default_rng(m * 131 + n)
    A = rng.integers(-50, 51, size=(m, n)).astype(np.float64)
    S = O.srht_explicit(3, s, m)
    assert np.array_equal(O.srht(3, s, A, scaled=False), S @ A)
    np.testing.assert_allclose(O.srht(3, s, A), S @ A / np.sqrt(s), rtol=0, atol=1e-12 * np.abs(A).sum())


def test_srht_exact_null_vector():
    # SAx = 0 exactly whenever Ax = 0 (integer A built with an integer null vector)
    rng = np.random.default_rng(2)
    m, n = 300, 6
    B = rng.integers(-20, 21, size=(m, n - 1)).astype(np.float64)
    z = rng.integers(-3, 4, size=n - 1).astype(np.float64)
    A = np.column_stack([B, B @ z])
    x = np.concatenate([z, [-1.0]])
    assert np.all(A @ x == 0)
    SA = O.srht(4, 64, A, scaled=False)
    assert np.all(SA @ x == 0)
    SA2 = O.sparse_sign(4, 64, 8, A, scaled=False)
    assert np.all(SA2 @ x == 0)


# ---------------------------------------------- H-RHT (Section 2) ----
def test_hash_rows_from_numpy_philox():
    # h[i], sg[i] from word (i mod 4) of stream-4 block i/4, drawn here with
    # numpy's Philox (counter (i/4, 0, 4, 0), key (seed, 0)) as a black box
    seed, s, mp = 77, 300, 64
    h, sg = O.hash_rows(seed, s, mp)
    for i in range(mp):
        ctr = np.array([i // 4 - 1 if i >= 4 else 2 ** 64 - 1, 0 if i >= 4 else 2 ** 64 - 1, 4 if i >= 4 else 3, 0],
                       dtype=np.uint64)
        w = int(np.random.Philox(counter=ctr, key=np.array([seed, 0], dtype=np.uint64)).random_raw(4)[i % 4])
        assert h[i] == ((w & 0xFFFFFFFF) * s) >> 32
        assert sg[i] == (-1 if w >> 63 else 1)


def test_hash_rows_uniform_and_balanced():
    s, mp = 64, 1 << 14
    h, sg = O.hash_rows(5, s, mp)
    assert h.min() >= 0 and h.max() < s
    assert scipy.stats.chisquare(np.bincount(h, minlength=s)).pvalue > 1e-4
    assert abs(sg.astype(np.int64).sum()) < 5 * np.sqrt(mp)
    assert not np.array_equal(h, O.hash_rows(6, s, mp)[0])


def test_hrht_is_hashing_times_scipy_hadamard():
    # S = S_h (1/sqrt m') H D with H from scipy and S_h one +-1 per column
    seed, m, s = 12, 45, 20
    lg = O.ceil_log2(m)
    mp = 1 << lg
    H = scipy.linalg.hadamard(mp).astype(np.float64)
    D = np.diag(O.signs(seed, mp).astype(np.float64))
    h, sg = O.hash_rows(seed, s, mp)
    Sh = np.zeros((s, mp))
    Sh[h, np.arange(mp)] = sg
    assert np.all(np.count_nonzero(Sh, axis=0) == 1)
    S_ref = (Sh @ H @ D)[:, :m]
    assert np.array_equal(O.hrht_explicit(seed, s, m), S_ref)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((m, 4))
    np.testing.assert_allclose(O.hrht(seed, s, A), S_ref @ A / np.sqrt(mp), rtol=0, atol=1e-13)


@pytest.mark.parametrize("m,n,s", [(64, 7, 32), (37, 5, 16), (1, 1, 1), (300, 3, 100), (4096, 2, 512)])
def test_hrht_matches_explicit_S_bitexact(m, n, s):
    rng = np.random.default_rng(m * 17 + n)
    A = rng.integers(-50, 51, size=(m, n)).astype(np.float64)
    S = O.hrht_explicit(8, s, m)
    assert np.array_equal(O.hrht(8, s, A, scaled=False), S @ A)


def test_hrht_exact_null_vector():
    rng = np.random.default_rng(4)
    m, n = 300, 6
    B = rng.integers(-20, 21, size=(m, n - 1)).astype(np.float64)
    z = rng.integers(-3, 4, size=n - 1).astype(np.float64)
    A = np.column_stack([B, B @ z])
    x = np.concatenate([z, [-1.0]])
    assert np.all(O.hrht(4, 64, A, scaled=False) @ x == 0)


def test_hrht_embeds_coherent_subspace_where_srht_fails():
    # Figure 1's difficult example: U = [I_n; 0], m = 1000, n = 100, s = 2n.
    # The Sylvester SRHT at s = 2n is no subspace embedding of span(U)
    # (sigma_min(S U) = 0: the sampled rows of H[:, :n] repeat), so Algorithm 1
    # returns a vector unrelated to the null vector; with the 1-hashing in place
    # of R, sigma(S U) lies in the Gaussian range and the solve succeeds, within
    # Theorem 3.2's bound.
    m, n, s = 1000, 100, 200
    U = np.zeros((m, n))
    U[:n, :n] = np.eye(n)
    V = workloads.orthonormal(np.random.default_rng(3), n, n)
    sig = np.concatenate([np.ones(n - 2), [0.1, 1e-6]])
    A = workloads.from_svd(U, sig, V)
    su_s = np.linalg.svd(O.srht(1, s, U), compute_uv=False)
    su_h = np.linalg.svd(O.hrht(1, s, U), compute_uv=False)
    assert su_s.min() < 1e-8
    assert 0.2 < su_h.min() and su_h.max() < 1.8
    bad = O.solve(O.SRHT, 1, s, A, 1)
    good = O.solve(O.HRHT, 1, s, A, 1)
    assert sine(V[:, -1:], bad["Vk"]) > 0.5
    R = np.linalg.qr(O.hrht(1, s, U), mode="r")
    bound = np.linalg.norm(R - np.linalg.inv(R).T, 2) / chi(good["sigk"][0] ** 2, sig[n - 2] ** 2)
    assert sine(V[:, -1:], good["Vk"]) <= bound * (1 + 1e-8) < 1e-4


# ------------------------------------------------------------ sparse sign ----
def test_sparse_sign_columns_structure():
    s, zeta, m = 50, 8, 4000
    rows, sg = O.sparse_sign_cols(21, s, zeta, m)
    assert rows.min() >= 0 and rows.max() < s
    for j in range(m):
        assert len(set(rows[j])) == zeta                  # distinct rows
    assert set(np.unique(sg)) == {-1, 1}
    # each row is hit uniformly (Floyd sampling gives a uniform zeta-subset)
    counts = np.bincount(rows.ravel(), minlength=s)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    assert abs(sg.astype(np.int64).sum()) < 5 * np.sqrt(m * zeta)


def test_sparse_sign_matches_explicit_bitexact():
    s, zeta, m, n = 24, 8, 60, 4
    rows, sg = O.sparse_sign_cols(3, s, zeta, m)
    S = np.zeros((s, m))
    for j in range(m):
        for i in range(zeta):
            S[rows[j, i], j] = sg[j, i]
    assert np.allclose(np.linalg.norm(S / np.sqrt(zeta), axis=0), 1.0)   # unit columns
    rng = np.random.default_rng(5)
    A = rng.integers(-30, 31, size=(m, n)).astype(np.float64)
    assert np.array_equal(O.sparse_sign(3, s, zeta, A, scaled=False), S @ A)


# --------------------------------------------------------------- Gaussian ----
def test_gaussian_entries_statistics():
    g = np.array([O.gaussian_entry(7, r, j) for r in range(64) for j in range(400)])
    assert abs(g.mean()) < 5 / np.sqrt(g.size)
    assert abs(g.var() - 1.0) < 5 * np.sqrt(2.0 / g.size)
    assert scipy.stats.kstest(g, "norm").pvalue > 1e-4


def test_gaussian_theorem_2_1_range():
    # Theorem 2.1: sqrt(s)-sqrt(n)-t <= sigma(G) <= sqrt(s)+sqrt(n)+t w.p. >= 1 - 2 exp(-t^2/2)
    s, n, t = 256, 32, 4.0
    G = np.array([[O.gaussian_entry(3, r, j) for j in range(n)] for r in range(s)])
    sv = np.linalg.svd(G, compute_uv=False)
    assert sv.max() <= np.sqrt(s) + np.sqrt(n) + t
    assert sv.min() >= np.sqrt(s) - np.sqrt(n) - t


def test_gaussian_sketch_equals_explicit():
    s, m, n = 16, 40, 3
    rng = np.random.default_rng(8)
    A = rng.standard_normal((m, n))
    G = np.array([[O.gaussian_entry(2, r, j) for j in range(m)] for r in range(s)])
    np.testing.assert_allclose(O.gaussian(2, s, A), G @ A / np.sqrt(s), rtol=1e-13, atol=1e-14)
    part = O.gaussian(2, s, A, cols=[2])
    np.testing.assert_allclose(part[:, 2], (G @ A / np.sqrt(s))[:, 2], rtol=1e-13, atol=1e-14)


def test_gaussian_rows_equal_explicit_product_and_full_sketch():
    # the sampled-rows routine against an explicit G A (brute force) and the
    # full sketch (same summation order: bit for bit); the term sizes against
    # their definition
    s, m, n = 24, 57, 4
    rng = np.random.default_rng(12)
    A = rng.standard_normal((m, n))
    G = np.array([[O.gaussian_entry(5, r, j) for j in range(m)] for r in range(s)])
    rows = [0, 7, 23, 7]
    out, mag = O.gaussian_rows(5, s, A, rows)
    np.testing.assert_allclose(out, (G @ A / np.sqrt(s))[rows], rtol=1e-13, atol=1e-14)
    assert np.array_equal(out, O.gaussian(5, s, A)[rows])
    want = np.sqrt(((G[rows][:, :, None] * A[None, :, :]) ** 2).sum(axis=1)) / np.sqrt(s)
    np.testing.assert_allclose(mag, want, rtol=1e-13)


# -------------------------------------------------------- QR and Jacobi ----
@pytest.mark.parametrize("s,n", [(40, 8), (128, 32), (9, 9), (5, 1)])
def test_householder_qr_against_lapack(s, n):
    rng = np.random.default_rng(s + n)
    B = rng.standard_normal((s, n))
    R = O.householder_qr_r(B)
    assert np.array_equal(np.triu(R), R)
    Rl = np.linalg.qr(B, mode="r")
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-12)
    # R^T R = B^T B, and Q = B R^{-1} is orthonormal
    np.testing.assert_allclose(R.T @ R, B.T @ B, atol=10 * s * U53 * np.linalg.norm(B) ** 2)
    Q = np.linalg.solve(R.T, B.T).T
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) < 10 * s * U53 * np.linalg.cond(B)


def test_householder_qr_zero_column():
    B = np.zeros((6, 3))
    B[:, 0] = 1.0
    B[:, 2] = np.arange(6)
    R = O.householder_qr_r(B)
    assert np.allclose(R.T @ R, B.T @ B)


@pytest.mark.parametrize("n", [1, 2, 17, 48])
def test_jacobi_against_lapack_svd(n):
    rng = np.random.default_rng(n)
    X0 = rng.standard_normal((n, n))
    X, V, sig, sweeps, st = O.jacobi(X0)
    assert st == O.OK and sweeps <= 15
    ref = np.linalg.svd(X0, compute_uv=False)
    np.testing.assert_allclose(np.sort(sig)[::-1], ref, rtol=1e-13 * n, atol=1e-15 * ref[0])
    # each column takes O(sweeps * n) rotations, each orthogonal to O(u); Frobenius adds sqrt(n)
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 10 * n ** 1.5 * U53
    np.testing.assert_allclose(X, X0 @ V, atol=50 * n * U53 * ref[0])
    # columns of X V are mutually orthogonal
    G = X.T @ X
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) <= 10 * n * U53 * ref[0] ** 2


def test_jacobi_graded_relative_accuracy():
    # column-graded R = R_s D with well-conditioned R_s: one-sided Jacobi gives
    # tiny singular values to high relative accuracy (Demmel & Veselic)
    rng = np.random.default_rng(4)
    n = 20
    Rs = np.linalg.qr(rng.standard_normal((n, n)))[0] + 0.1 * rng.standard_normal((n, n))
    D = np.diag(np.logspace(0, -14, n))
    X0 = Rs @ D
    _, _, sig, _, st = O.jacobi(X0)
    assert st == O.OK
    # reference via the well-conditioned factor: sigma(X0) = sigma(Rs D); compare
    # against LAPACK on the scaled problem computed in extended steps
    ref = np.linalg.svd(X0, compute_uv=False)
    kappa = np.linalg.cond(Rs)
    rel = np.abs(np.sort(sig)[::-1] - ref) / ref
    # LAPACK's own relative error on tiny values can be ~ u*sigma_1/sigma_i;
    # the product of all sigma equals |det X0| = |det Rs| prod(D) exactly in theory
    logdet = np.sum(np.log(sig))
    ref_logdet = np.linalg.slogdet(Rs)[1] + np.sum(np.log(np.diag(D)))
    assert abs(logdet - ref_logdet) < 1e-10 * n * kappa
    assert rel[:5].max() < 1e-12


def test_jacobi_reports_noconv():
    rng = np.random.default_rng(3)
    X0 = rng.standard_normal((30, 30))
    _, _, _, sweeps, st = O.jacobi(X0, max_sweeps=1)
    assert st == O.ERR_NOCONV and sweeps == 1


def test_extract_order_and_sign():
    sig = np.array([3.0, 1.0, 2.0, 1.0])
    V = np.eye(4)
    V[:, 1] *= -1
    Vk, sk, order = O.extract(sig, V, 2)
    assert list(order) == [0, 2, 1, 3]
    assert list(sk) == [1.0, 1.0]
    assert np.array_equal(Vk[:, 0], np.eye(4)[:, 1])     # sign flipped to positive max entry
    assert np.array_equal(Vk[:, 1], np.eye(4)[:, 3])


def test_residual_against_numpy():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((50, 6))
    W = rng.standard_normal((6, 2))
    assert abs(O.residual(A, W) - np.linalg.norm(A @ W)) < 1e-12 * np.linalg.norm(A @ W)


# ------------------------------------------- whole solve (Algorithm 1) ----
@pytest.mark.parametrize("kind", [O.SRHT, O.HRHT, O.SPARSE_SIGN, O.GAUSSIAN])
def test_ostrowski_bracket(kind):
    # proof of Theorem 2.3: sigma_min(S U_A) sigma_i(A) <= sigma_i(SA) <= sigma_max(S U_A) sigma_i(A)
    # for the realized S of every sketch kind
    w = workloads.plain(seed=3, m=1024, n=16)
    A, s = w["A"], 64
    SA = O.sketch(kind, 5, s, A)
    UA, sa, _ = np.linalg.svd(A, full_matrices=False)
    SU = O.sketch(kind, 5, s, UA)
    su = np.linalg.svd(SU, compute_uv=False)
    ssa = np.linalg.svd(SA, compute_uv=False)
    slack = 1e-12
    assert np.all(ssa <= su.max() * sa * (1 + slack) + 1e-15)
    # lower bracket (relative, on values far from rounding level)
    big = sa > 1e-8
    assert np.all(ssa[big] >= su.min() * sa[big] * (1 - slack))


@pytest.mark.parametrize("kind", [O.SRHT, O.GAUSSIAN, O.SPARSE_SIGN, O.HRHT])
def test_theorem_3_2_bound_deterministic(kind):
    # Figure-1 style input: m=1000, n=100, k=1, sigma = (1,...,1, 0.1, sigma_n)
    rng = np.random.default_rng(10 + kind)
    m, n, s = 1000, 100, 400
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.ones(n - 2), [0.1, 1e-5]])
    A = workloads.from_svd(U, sig, V)
    out = O.solve(kind, 17, s, A, 1)
    # realized X^* U = S U and its R factor
    SU = O.sketch(kind, 17, s, U)
    R = np.linalg.qr(SU, mode="r")
    Mnorm = np.linalg.norm(R - np.linalg.inv(R).T, 2)
    alpha = out["sigk"][0]                 # tilde sigma_n
    alpha_delta = sig[n - 2]               # sigma_{n-1}
    assert alpha_delta > alpha
    bound = Mnorm / chi(alpha ** 2, alpha_delta ** 2)
    s_true = sine(V[:, -1:], out["Vk"])
    assert s_true <= bound * (1 + 1e-8) + 1e-15
    # residual: ||A W~||_F <= kappa(S U) ||A W||_F (proof of Theorem 2.3 before its constants)
    su = np.linalg.svd(SU, compute_uv=False)
    assert O.residual(A, out["Vk"]) <= su.max() / su.min() * sig[-1] * (1 + 1e-6)


@pytest.mark.parametrize("kind", [O.SRHT, O.GAUSSIAN, O.SPARSE_SIGN, O.HRHT])
def test_theorem_3_4_bounds_deterministic(kind):
    # Subspaces of different dimensions (Theorem 3.4): the trailing k = 4 singular
    # values of A are 1e-2 .. 1e-3 with no gap among them, so the trailing l = 2
    # alone are not determined, but the theorem still places
    #   case 1: the sketched trailing l inside A's trailing k,
    #   case 2: A's trailing l inside the sketched trailing k,
    # both within ||R - R^{-T}||_2 / chi(alpha^2, (alpha + delta)^2), R from S U.
    rng = np.random.default_rng(40 + kind)
    m, n, s, k, l = 1000, 100, 400, 4, 2
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.ones(n - k), np.logspace(-2, -3, k)])
    A = workloads.from_svd(U, sig, V)
    out = O.solve(kind, 23, s, A, k)
    assert np.all(np.diff(out["sigk"]) <= 0)  # tilde sigma_{n-k+1} >= ... >= tilde sigma_n
    st = np.sort(out["sigma"])[::-1]         # tilde sigma_1 >= ... >= tilde sigma_n
    R = np.linalg.qr(O.sketch(kind, 23, s, U), mode="r")
    Mnorm = np.linalg.norm(R - np.linalg.inv(R).T, 2)
    Vl = out["Vk"][:, k - l:]                # the trailing l sketched vectors
    # case 1: alpha = tilde sigma_{n-l+1}, alpha + delta = sigma_{n-k}
    alpha, ad = st[n - l], sig[n - k - 1]
    assert ad > alpha
    b1 = Mnorm / chi(alpha ** 2, ad ** 2)
    assert sine(V[:, n - k:], Vl) <= b1 * (1 + 1e-8) + 1e-15
    # case 2: alpha = sigma_{n-l+1}, alpha + delta = tilde sigma_{n-k}
    alpha, ad = sig[n - l], st[n - k - 1]
    assert ad > alpha
    b2 = Mnorm / chi(alpha ** 2, ad ** 2)
    assert sine(out["Vk"], V[:, n - l:]) <= b2 * (1 + 1e-8) + 1e-15
    # the bounds are informative here (sigma_{n-k} / sigma_{n-l+1} ~ 300), so a
    # window shifted onto a sigma = 1 direction fails them
    assert max(b1, b2) < 0.05


def test_exact_null_space_preserved():
    # sigma_{n-k+1..n} = 0: the sketched trailing subspace is the null space (Section 3.1.1)
    rng = np.random.default_rng(6)
    m, n, k = 2048, 24, 3
    B = rng.standard_normal((m, n - k))
    Z = rng.standard_normal((n - k, k))
    A = np.asfortranarray(np.column_stack([B, B @ Z]))
    N = np.vstack([Z, -np.eye(k)])            # A N = 0 up to rounding of B @ Z
    for kind in (O.SRHT, O.SPARSE_SIGN, O.GAUSSIAN, O.HRHT):
        out = O.solve(kind, 1, 4 * n, A, k)
        assert sine(N, out["Vk"]) < 1e-12
        assert O.residual(A, out["Vk"]) < 1e-13 * np.linalg.norm(A)


def test_plain_workload_a_priori_bound():
    # m=4096, n=32: a-priori bound of Section 3.1.1 with sigma_31 = 1e-4, sigma_32 = 1e-12
    w = workloads.plain(seed=0)
    out = O.solve(O.SRHT, 0, w["s"], w["A"], 1)
    sn1, sn = w["sigma"][-2], w["sigma"][-1]
    apriori = 3.36 * sn1 * sn / (sn1 ** 2 - 2.56 * sn ** 2)
    assert sine(w["V"][:, -1:], out["Vk"]) <= max(apriori, 1e-11)
    # Ostrowski on sigma_n from the realized sketch
    SU = O.srht(0, w["s"], w["U"])
    su = np.linalg.svd(SU, compute_uv=False)
    assert su.min() * sn * (1 - 1e-3) <= out["sigk"][0] <= su.max() * sn * (1 + 1e-3)


def test_solve_matches_lapack_svd_of_sketch():
    # SVD(SA) and SVD(R) share sigma and V (proof of Theorem 3.2)
    w = workloads.graded(seed=1, m=2000, n=40, k=2)
    out = O.solve(O.SRHT, 3, 160, w["A"], 2)
    _, sv, Vt = np.linalg.svd(out["SA"])
    np.testing.assert_allclose(np.sort(out["sigma"])[::-1], sv, rtol=1e-9, atol=1e-15)
    assert sine(Vt.T[:, -2:], out["Vk"]) < 1e-8


# --------------------------------------------------- TLS (Section 4) ----
def test_tls_against_dense_svd():
    rng = np.random.default_rng(12)
    m, n = 4096, 20
    Xb, x_true = workloads.tls_problem(rng, m, n, noise=1e-3)
    x, v, st = O.tls(5, 2 * (n + 1), Xb)
    assert st == O.OK
    Vd = np.linalg.svd(Xb)[2].T[:, -1]
    x_dense = -Vd[:n] / Vd[n]
    # relative error of the sketched TLS solution is O(sigma_{n+1}/sigma_n) (Section 4)
    sv = np.linalg.svd(Xb, compute_uv=False)
    gap = sv[n] / np.linalg.svd(Xb[:, :n], compute_uv=False)[-1]
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 50 * gap
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) < 1e-2


def test_tls_no_solution_flag():
    m, n = 256, 4
    rng = np.random.default_rng(1)
    X = rng.standard_normal((m, n))
    X[:, 3] = X[:, 2]                     # null vector e3 - e4 has zero last entry
    Xb = np.column_stack([X, rng.standard_normal(m)])
    _, _, st = O.tls(1, 2 * (n + 1), Xb)
    assert st == O.ERR_TLS_NOSOLUTION


# --------------------------------------- updating/downdating (Section 5) ----
def test_row_downdate_identity_and_closed_form():
    rng = np.random.default_rng(2)
    m, n, s = 200, 5, 32
    A = rng.integers(-9, 10, size=(m, n)).astype(np.float64)
    S = O.srht_explicit(7, s, m)
    SA = O.srht(7, s, A, scaled=False)
    for j in (0, 17, 199):
        e = np.zeros((m, 1))
        e[j] = 1.0
        Se = O.srht(7, s, e, scaled=False)[:, 0]
        assert np.array_equal(Se, S[:, j])                 # sketch of e_j = column j of S
        Aj = A.copy()
        Aj[j, :] = 0.0
        # Algorithm 3: S_j A_j = SA - S(:, j) A(j, :)
        assert np.array_equal(O.srht(7, s, Aj, scaled=False), SA - np.outer(Se, A[j]))


def test_row_update_identity_gaussian():
    # Algorithm 2: appending row a_{m+1} and column g/sqrt(s) to S adds g a_{m+1}/sqrt(s)
    rng = np.random.default_rng(4)
    m, n, s = 30, 3, 8
    A = rng.standard_normal((m + 1, n))
    G = np.array([[O.gaussian_entry(5, r, j) for j in range(m + 1)] for r in range(s)])
    SA_m = G[:, :m] @ A[:m] / np.sqrt(s)
    SA_full = O.gaussian(5, s, A)
    np.testing.assert_allclose(SA_full, SA_m + np.outer(G[:, m], A[m]) / np.sqrt(s), atol=1e-13)


# ----------------------------------------------------- AAA (Section 6) ----
def test_aaa_incremental_sketch_equals_fresh_sketch():
    x, f = workloads.aaa_points(seed=1, m=600, scale=10.0)
    K, smax = 8, 32
    sup, W, err, st, SAk = O.aaa(3, x, f, K, smax, return_sketch=True)
    assert len(set(sup.tolist())) == K
    # Loewner matrix of the final support set, support rows zeroed
    L = np.zeros((x.size, K))
    for l, jl in enumerate(sup):
        with np.errstate(divide="ignore", invalid="ignore"):
            L[:, l] = (f - f[jl]) / (x - x[jl])
    L[sup, :] = 0.0
    np.testing.assert_allclose(SAk, O.srht(3, smax, L), atol=1e-12 * np.abs(L).max() * np.sqrt(x.size))


def test_aaa_converges_on_tanh():
    x, f = workloads.aaa_points(seed=0, m=4000, scale=50.0)
    sup, W, err, st = O.aaa(1, x, f, 40, 160)
    assert st == O.OK
    assert err[-1] < 1e-10 * np.abs(f).max()
    # interpolation at support points: each weight vector is a unit vector
    for k in range(1, 41):
        np.testing.assert_allclose(np.linalg.norm(W[k - 1, :k]), 1.0, rtol=1e-12)


def test_aaa_teacher_forcing_reproduces_free_run():
    x, f = workloads.aaa_points(seed=2, m=1000, scale=20.0)
    sup, W, err, st = O.aaa(4, x, f, 12, 48)
    sup2, W2, err2, st2 = O.aaa(4, x, f, 12, 48, forced=sup)
    assert np.array_equal(sup, sup2) and np.array_equal(W, W2) and np.array_equal(err, err2)


# ------------------------------------------------------------ adjoint ----
def _loss_and_grad(Vk, W):
    P = Vk @ Vk.T
    L = np.linalg.norm(P @ W) ** 2
    return L, 2.0 * W @ W.T @ Vk


def test_backward_finite_differences():
    rng = np.random.default_rng(7)
    m, n, k, s = 512, 12, 3, 48
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.linspace(3, 1, n - k), [1e-3, 7e-4, 4e-4]])
    A = workloads.from_svd(U, sig, V)
    Wl = rng.standard_normal((n, 4))
    out = O.solve(O.SRHT, 9, s, A, k)
    _, dV = _loss_and_grad(out["Vk"], Wl)
    dA = O.backward_srht(9, s, m, out["SA"], out["V"], out["sigma"], out["Vk"], dV)
    h = 1e-6
    for d in range(3):
        E = np.asfortranarray(rng.standard_normal((m, n)))
        Lp = _loss_and_grad(O.solve(O.SRHT, 9, s, A + h * E, k)["Vk"], Wl)[0]
        Lm = _loss_and_grad(O.solve(O.SRHT, 9, s, A - h * E, k)["Vk"], Wl)[0]
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(dA * E))
        assert abs(an - fd) <= 1e-6 * abs(fd) + 1e-9


def test_backward_against_torch_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    m, n, k, s = 128, 10, 2, 40
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.linspace(2, 1, n - k), [1e-2, 5e-3]])
    A = workloads.from_svd(U, sig, V)
    Wl = rng.standard_normal((n, 3))
    S = O.srht_explicit(2, s, m) / np.sqrt(s)
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    St = torch.tensor(S, dtype=torch.float64)
    _, _, Vh = torch.linalg.svd(St @ At, full_matrices=False)
    Vk_t = Vh.T[:, -k:]
    P = Vk_t @ Vk_t.T
    L = torch.linalg.norm(P @ torch.tensor(Wl)) ** 2
    L.backward()
    out = O.solve(O.SRHT, 2, s, A, k)
    _, dV = _loss_and_grad(out["Vk"], Wl)
    dA = O.backward_srht(2, s, m, out["SA"], out["V"], out["sigma"], out["Vk"], dV)
    ref = At.grad.numpy()
    assert np.linalg.norm(dA - ref) <= 1e-8 * np.linalg.norm(ref)


def test_backward_gauge_invariance():
    # the adjoint ignores the components of dL/dV_k along span(V_k) and is
    # unchanged by flipping the sign of a returned vector with its gradient
    rng = np.random.default_rng(9)
    m, n, k, s = 256, 8, 2, 32
    A = np.asfortranarray(rng.standard_normal((m, n)))
    out = O.solve(O.SRHT, 1, s, A, k)
    Wl = rng.standard_normal((n, 2))
    _, dV = _loss_and_grad(out["Vk"], Wl)
    dA1 = O.backward_srht(1, s, m, out["SA"], out["V"], out["sigma"], out["Vk"], dV)
    K = rng.standard_normal((k, k))
    dA2 = O.backward_srht(1, s, m, out["SA"], out["V"], out["sigma"], out["Vk"], dV + out["Vk"] @ K)
    assert np.linalg.norm(dA1 - dA2) <= 1e-12 * np.linalg.norm(dA1)
    flip = np.array([1.0, -1.0])
    dA3 = O.backward_srht(1, s, m, out["SA"], out["V"], out["sigma"], out["Vk"] * flip, dV * flip)
    assert np.linalg.norm(dA1 - dA3) <= 1e-12 * np.linalg.norm(dA1)


# --------------------------------------------------- tolerance version ----
def test_solve_eps_finds_the_exact_null_space():
    # Section 2, after Algorithm 1: with sigma(A) = (1 .. 1e-3, 0, 0, 0) the
    # sketch keeps the three exact zeros (SA x = 0 whenever A x = 0) and the
    # nonzero values within a constant factor, so eps = 1e-8 selects exactly 3
    # vectors, and they annihilate A.
    w = workloads.at_scale(seed=3, m=2048, n=24, null_dim=3)
    A = w["A"]
    Vk, sk, k, full = O.solve_eps(O.SRHT, 0, 96, A, 1e-8)
    assert k == 3
    assert np.all(sk < 1e-8)
    assert np.linalg.norm(A @ Vk) <= 1e-13 * np.linalg.norm(A)
    assert sine(w["V"][:, -3:], Vk) < 1e-10
    # the same vectors, order and signs as the fixed-k solve
    ref = O.solve(O.SRHT, 0, 96, A, 3)
    np.testing.assert_array_equal(Vk, ref["Vk"])
    np.testing.assert_array_equal(sk, ref["sigk"])


def test_solve_eps_limits():
    # eps = 0 selects nothing (singular values are >= 0); eps above sigma_1
    # selects everything: W is then all of V, orthonormal
    w = workloads.plain(seed=1, m=512, n=12)
    A = w["A"]
    _, _, k0, _ = O.solve_eps(O.SRHT, 0, 48, A, 0.0)
    assert k0 == 0
    Vk, sk, kn, full = O.solve_eps(O.SRHT, 0, 48, A, 2.0 * np.linalg.norm(A, 2) * 2)
    assert kn == 12
    assert np.all(np.diff(sk) <= 0)  # non-increasing, the smallest last
    np.testing.assert_allclose(Vk.T @ Vk, np.eye(12), atol=1e-13)


# ------------------------------------------------------ row updates (Section 5) ----
@pytest.mark.parametrize("kind", [O.SRHT, O.SPARSE_SIGN, O.GAUSSIAN])
def test_row_remove_equals_sketch_with_row_zeroed(kind):
    # Removing row j from the sketch is sketching A with row j set to zero
    # (Section 5: removing column j of S zeroes row j's contribution).  This
    # pins the regenerated column S e_j against the full sketch.
    rng = np.random.default_rng(kind + 7)
    m, n, s, j = 700, 5, 64, 333
    A = np.asfortranarray(rng.standard_normal((m, n)))
    SA = O.sketch(kind, 5, s, A, zeta=8)
    upd = O.sketch_update(kind, 5, s, SA, m, 1, j, A[j, :], zeta=8)
    A0 = A.copy(order="F")
    A0[j, :] = 0.0
    ref = O.sketch(kind, 5, s, A0, zeta=8)
    np.testing.assert_allclose(upd, ref, rtol=0, atol=1e-13 * np.linalg.norm(SA))


def test_gaussian_row_append_equals_sketch_of_grown_matrix():
    # Algorithm 2: [G | g_{m+1}] is the Gaussian sketch of m + 1 rows, so the
    # updated sketch equals the Gaussian sketch of [A; a].
    rng = np.random.default_rng(3)
    m, n, s = 301, 4, 32
    A = np.asfortranarray(rng.standard_normal((m, n)))
    a = rng.standard_normal(n)
    SA = O.sketch(O.GAUSSIAN, 11, s, A)
    upd = O.sketch_update(O.GAUSSIAN, 11, s, SA, m, 0, m, a)
    ref = O.sketch(O.GAUSSIAN, 11, s, np.asfortranarray(np.vstack([A, a[None, :]])))
    np.testing.assert_allclose(upd, ref, rtol=0, atol=1e-13 * np.linalg.norm(ref))


@pytest.mark.parametrize("kind", [O.SRHT, O.SPARSE_SIGN])
def test_row_append_then_remove_restores(kind):
    rng = np.random.default_rng(kind + 20)
    m, n, s = 900, 3, 48
    A = np.asfortranarray(rng.standard_normal((m, n)))
    SA = O.sketch(kind, 2, s, A, zeta=8)
    a = rng.standard_normal(n)
    up = O.sketch_update(kind, 2, s, SA, m, 0, m + 4, a, zeta=8)
    assert np.linalg.norm(up - SA) > 0.1 * np.linalg.norm(a)
    back = O.sketch_update(kind, 2, s, up, m, 1, m + 4, a, zeta=8)
    np.testing.assert_allclose(back, SA, rtol=0, atol=1e-13 * np.linalg.norm(SA))
