"""GPU dense stage (lines 3-4 of Algorithm 1 on a given sketch) against the
oracle's Householder QR + one-sided Jacobi on the same SA.

The GPU preconditions with two QRs and orders the Jacobi pairs differently
(cluster ring), so results agree up to rounding, not bit for bit: singular
values to relative 1e-12 of sigma_1 (absolute) and 1e-9 (relative, where
sigma_i / sigma_1 > 1e-6), the trailing subspace by its sine when the gap
allows (u sigma_1 / gap <= 1e-10), and V orthonormal to 1e-13.
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_00975_gb300 import workloads
from tests.helpers import sine

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_00975_gb300 import build
    build.build()
    from paper_2206_00975_gb300 import api as a
    return a


def sketch_like(seed, s, n, null_dim):
    # SA = Q diag(sigma) V^T with sigma log-spaced 1..1e-5 and null_dim zeros
    rng = np.random.default_rng(seed)
    Q = workloads.orthonormal(rng, s, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.logspace(0, -5, n - null_dim), np.zeros(null_dim)])
    return np.asfortranarray(workloads.from_svd(Q, sig, V)), V, sig


@pytest.mark.parametrize("s,n,k", [(1024, 256, 4), (400, 100, 3), (68, 17, 2), (512, 250, 5), (64, 16, 1)])
def test_dense_stage_parity(api, s, n, k):
    SA, Vtrue, sig = sketch_like(s + n, s, n, k)
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    ws = api.workspace(d, s, n, k, "cuda")
    Vk, sk, sv, status = api.ns_solve_sketched(d, api.colmajor(SA, device="cuda"), k, save=True, ws=ws)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    stats = api.jacobi_stats(d, s, n, ws, sketched=True)
    assert stats[3] in (8, 16), "the cluster-ring Jacobi should run for n <= 256"
    if n >= 64:   # the FP32 linear phase ran, and the FP64 iteration only finished it
        assert stats[4] >= 1 and stats[5] > 0, stats
        assert stats[0] <= 3, stats
    Vk_or, sk_or, V_or, sig_or, _, st = O.solve_sketched(SA, k)
    assert st == 0
    _, V, sigma = api.unpack_save(sv, s, n)
    V = V.cpu().numpy()
    sigma = np.sort(sigma.cpu().numpy())[::-1]
    s1 = sig_or.max()
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-13 * n
    ref = np.sort(sig_or)[::-1]
    assert np.max(np.abs(sigma - ref)) <= 1e-12 * s1
    big = ref > 1e-6 * s1
    assert np.max(np.abs(sigma[big] - ref[big]) / ref[big]) <= 1e-9
    # trailing subspace (exact zeros: gap sigma_{n-k} = 1e-5 sigma_1)
    gap = ref[n - k - 1] - ref[n - k]
    assert U53 * s1 / gap <= 1e-10
    assert sine(Vk_or, Vk.cpu().numpy()) < 1e-8
    assert sine(Vtrue[:, -k:], Vk.cpu().numpy()) < 1e-8


def test_dense_stage_repeatable(api):
    # the same sketch twice in a row through the same workspace: identical bits
    SA, _, _ = sketch_like(5, 1024, 256, 4)
    d = api.desc(api.NS_SRHT, s=1024, seed=0)
    ws = api.workspace(d, 1024, 256, 4, "cuda")
    SAd = api.colmajor(SA, device="cuda")
    a = api.ns_solve_sketched(d, SAd, 4, ws=ws)[0].clone()
    b = api.ns_solve_sketched(d, SAd, 4, ws=ws)[0]
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_dense_stage_wide_range(api):
    # a full-rank sketch (sigma 1 .. 1e-5) with column scales spanning 1e-60 ..
    # 1e60: one-sided Jacobi determines every singular value to high relative
    # accuracy here (the column-equilibrated matrix has condition ~1e5), so the
    # static norm ordering before the unpivoted QR must keep it, and the FP32
    # images of the scaled sums and the tiny-angle path must keep converging.
    # (Far wider ranges make the products alpha beta of the threshold test
    # underflow, and plain one-sided Jacobi, the oracle's included, stalls.)
    rng = np.random.default_rng(11)
    s, n, k = 256, 48, 2
    Q = workloads.orthonormal(rng, s, n)
    V = workloads.orthonormal(rng, n, n)
    SA = workloads.from_svd(Q, np.logspace(0, -5, n), V)
    D = np.logspace(-60, 60, n)
    SAs = np.asfortranarray(SA * D[None, :])
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    Vk, sk, sv, status = api.ns_solve_sketched(d, api.colmajor(SAs, device="cuda"), k, save=True)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Vk_or, sk_or, _, sig_or, _, st = O.solve_sketched(SAs, k)
    assert st == 0
    _, _, sigma = api.unpack_save(sv, s, n)
    np.testing.assert_allclose(np.sort(sigma.cpu().numpy()), np.sort(sig_or), rtol=1e-8, atol=0)
    np.testing.assert_allclose(sk.cpu().numpy(), sk_or, rtol=1e-8, atol=0)


def test_dense_stage_near_repeated_column(api):
    # Two columns parallel to ~1e-9: they sit next to each other in the
    # decreasing-norm order, so when the owner of the second applies the
    # first one's reflector, the downdated tail norm cancels to ~1e-18 of its
    # terms and is recomputed from the updated column.
    rng = np.random.default_rng(21)
    s, n, k = 400, 100, 1
    SA = rng.standard_normal((s, n))
    SA[:, 7] = SA[:, 3] + 1e-9 * rng.standard_normal(s)
    order = np.argsort(-np.sum(SA * SA, axis=0), kind="stable")
    pos = sorted([int(np.where(order == 3)[0][0]), int(np.where(order == 7)[0][0])])
    assert pos[1] == pos[0] + 1 and pos[0] >= 1  # adjacent, past the first reflector
    SA = np.asfortranarray(SA)
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    Vk, sk, sv, status = api.ns_solve_sketched(d, api.colmajor(SA, device="cuda"), k, save=True)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Vk_or, sk_or, _, sig_or, _, st = O.solve_sketched(SA, k)
    assert st == 0
    _, V, sigma = api.unpack_save(sv, s, n)
    V = V.cpu().numpy()
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-13 * n
    s1 = sig_or.max()
    np.testing.assert_allclose(np.sort(sigma.cpu().numpy()), np.sort(sig_or), rtol=0, atol=1e-12 * s1)
    assert sine(Vk_or, Vk.cpu().numpy()) < 1e-8


def test_dense_stage_fp32_phase_guard(api):
    # 100 columns graded over 1 .. 1e-8 take part in the FP32 phase; 28 more,
    # graded from 1e-20 down to 1e-60 (not null: sigma of high relative accuracy),
    # are left out of it (below 2^-60 of the largest norm).  Every singular
    # value must keep one-sided Jacobi's relative accuracy.
    rng = np.random.default_rng(19)
    s, n, k = 512, 128, 2
    Q = workloads.orthonormal(rng, s, n)
    V = workloads.orthonormal(rng, n, n)
    SA = workloads.from_svd(Q, np.logspace(0, -3, n), V)
    D = np.concatenate([np.logspace(0, -8, 100), np.logspace(-20, -60, 28)])
    SAs = np.asfortranarray(SA * D[None, :])
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    ws = api.workspace(d, s, n, k, "cuda")
    Vk, sk, sv, status = api.ns_solve_sketched(d, api.colmajor(SAs, device="cuda"), k, save=True, ws=ws)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    stats = api.jacobi_stats(d, s, n, ws, sketched=True)
    assert stats[4] >= 1, stats   # the phase ran on the 100 leading columns
    Vk_or, sk_or, _, sig_or, _, st = O.solve_sketched(SAs, k)
    assert st == 0
    _, V, sigma = api.unpack_save(sv, s, n)
    V = V.cpu().numpy()
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-13 * n
    np.testing.assert_allclose(np.sort(sigma.cpu().numpy()), np.sort(sig_or), rtol=1e-8, atol=0)
    np.testing.assert_allclose(sk.cpu().numpy(), sk_or, rtol=1e-8, atol=0)


def test_dense_stage_benchmark_spectrum(api):
    # the benchmark's dense problem (sigma log-spaced 1 .. 1e-6 and a 4-dimensional
    # exact null space, n = 256, s = 1024), which runs the FP32 phase: it must
    # not cost accuracy against the oracle (relative 1e-9 down to 1e-6 sigma_1)
    rng = np.random.default_rng(23)
    s, n, k = 1024, 256, 4
    Q = workloads.orthonormal(rng, s, n)
    Vt = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.logspace(0, -6, n - k), np.zeros(k)])
    SA = np.asfortranarray(workloads.from_svd(Q, sig, Vt))
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    ws = api.workspace(d, s, n, k, "cuda")
    Vk, sk, sv, status = api.ns_solve_sketched(d, api.colmajor(SA, device="cuda"), k, save=True, ws=ws)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    stats = api.jacobi_stats(d, s, n, ws, sketched=True)
    print("benchmark spectrum: FP64 sweeps %d rotations %d checks %d; FP32 sweeps %d rotations %d" %
          (stats[0], stats[1], stats[2], stats[4], stats[5]))
    # after the FP32 phase and two first-order completions the FP64 iteration
    # needs at most its convergence check and one sweep
    assert stats[4] >= 1 and stats[0] <= 1, stats
    Vk_or, sk_or, _, sig_or, _, st = O.solve_sketched(SA, k)
    _, V, sigma = api.unpack_save(sv, s, n)
    V = V.cpu().numpy()
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-13 * n
    ref = np.sort(sig_or)[::-1]
    got = np.sort(sigma.cpu().numpy())[::-1]
    assert np.max(np.abs(got - ref)) <= 1e-12 * ref[0]
    big = ref > 1e-6 * ref[0] * 0.999
    assert np.max(np.abs(got[big] - ref[big]) / ref[big]) <= 1e-9
    assert sine(Vk_or, Vk.cpu().numpy()) < 1e-8
    assert sine(Vt[:, -k:], Vk.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("kind", ["clustered", "half_null"])
def test_dense_stage_completion_guard(api, kind):
    # The first-order completion after the FP32 phase, on spectra where it must
    # hold back: pairs of singular values 1e-10 apart (their rotations are far
    # from small, so those pairs are left to the FP64 sweeps), and a
    # 128-dimensional null space (the FP32 phase stops after one sweep, the
    # cosines are still large and the step is scaled down).  V stays
    # orthonormal, sigma accurate, and the computed null vectors annihilate SA.
    rng = np.random.default_rng(31)
    s, n, k = 1024, 256, 4
    Q = workloads.orthonormal(rng, s, n)
    Vt = workloads.orthonormal(rng, n, n)
    if kind == "clustered":
        base = np.logspace(0, -5, (n - k) // 2)
        sig = np.concatenate([np.sort(np.concatenate([base, base * (1 + 1e-10)]))[::-1], np.zeros(k)])
    else:
        sig = np.concatenate([np.logspace(0, -3, n // 2), np.zeros(n // 2)])
    SA = np.asfortranarray(workloads.from_svd(Q, sig, Vt))
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    ws = api.workspace(d, s, n, k, "cuda")
    Vk, sk, sv, status = api.ns_solve_sketched(d, api.colmajor(SA, device="cuda"), k, save=True, ws=ws)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    stats = api.jacobi_stats(d, s, n, ws, sketched=True)
    assert stats[4] >= 1, stats
    _, V, sigma = api.unpack_save(sv, s, n)
    V = V.cpu().numpy()
    assert np.linalg.norm(V.T @ V - np.eye(n)) < 1e-13 * n
    _, _, _, sig_or, _, st = O.solve_sketched(SA, k)
    assert st == 0
    ref = np.sort(sig_or)[::-1]
    got = np.sort(sigma.cpu().numpy())[::-1]
    assert np.max(np.abs(got - ref)) <= 1e-12 * ref[0]
    Vkn = Vk.cpu().numpy()
    assert np.linalg.norm(SA @ Vkn) <= 1e-13 * n * ref[0]
    if kind == "clustered":
        assert sine(Vt[:, -k:], Vkn) < 1e-8
