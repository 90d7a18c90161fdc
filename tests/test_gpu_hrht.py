"""GPU parity of the H-RHT sketch (Section 2: the SRFT with its restriction
replaced by a 1-hashing matrix) against the oracle.

Tolerances:
  * integer inputs: bit-exact (both sides are exact on them: the GPU's two
    roundings, onto its block quantum and onto the column quantum, drop only
    zero bits, and the oracle's FP64 sums stay below 2^53);
  * FP64 inputs: |SA - SA_oracle| <= 2^-40 max |SA_oracle(:, c)| per column.
    The GPU rounds each transformed block value once onto 2^-P of the
    column's largest (P >= 44 at these sizes) and sums exactly, so its error is
    below B cmax 2^-P of the largest |Z| (B blocks, cmax rows per bucket);
    the measured error is ~1e-14 of the column's largest entry;
  * solve on Figure 1's coherent example: the H-RHT's trailing vector within
    Theorem 3.2's bound on the realized S, and the oracle's to 1e-8, where the
    SRHT at the same s fails.
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_00975_gb300 import workloads
from tests.helpers import chi, sine

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_00975_gb300 import build
    build.build()
    from paper_2206_00975_gb300 import api as a
    return a


def sketch(api, A, s, seed):
    d = api.desc(api.NS_HRHT, s=s, seed=seed)
    SA = api.ns_sketch(d, api.colmajor(np.asfortranarray(A), device="cuda"))
    torch.cuda.synchronize()
    return SA.cpu().numpy()


@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (2, 1, 2), (3, 2, 3), (1000, 3, 200), (4095, 2, 100), (4096, 5, 512),
                                   (5000, 4, 300), (70000, 3, 700), ((1 << 18) + 3, 2, 2048)])
def test_hrht_integer_inputs_bitexact(api, m, n, s):
    rng = np.random.default_rng(m + 3 * n)
    A = rng.integers(-50, 51, size=(m, n)).astype(np.float64)
    assert np.array_equal(sketch(api, A, s, 9), O.hrht(9, s, A))


@pytest.mark.parametrize("m", [(1 << 20) + 1, (1 << 21) + 1, (1 << 22) + 1, (1 << 23) + 1])
def test_hrht_three_phase_geometries_bitexact(api, m):
    # m' = 2^21 .. 2^24: 512 .. 4096 blocks across, so the cross-block
    # transform takes three register phases, and at 2048 and 4096 blocks the
    # slab is 2 and 1 values wide (8- and 4-byte staged copies)
    rng = np.random.default_rng(m)
    A = rng.integers(-50, 51, size=(m, 1)).astype(np.float64)
    assert np.array_equal(sketch(api, A, 1000, 13), O.hrht(13, 1000, A))


@pytest.mark.parametrize("m,n,s", [(37, 3, 16), (1000, 16, 128), (4097, 6, 640), ((1 << 14) + 3, 8, 500),
                                   (1 << 17, 4, 1000), (3 * 4096 + 17, 3, 4096), (20000, 2, 16000)])
def test_hrht_sketch_parity(api, m, n, s):
    # (the last case, s = 16000, takes the single-stage pass 2: two stages of
    # staged tiles and the s accumulators would not fit in shared memory)
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-3, 3, size=(1, n)))
    got = sketch(api, A, s, 4)
    ref = O.hrht(4, s, A)
    for c in range(n):
        assert np.max(np.abs(got[:, c] - ref[:, c])) <= 2.0 ** -40 * np.max(np.abs(ref[:, c]))


@pytest.mark.parametrize("m,n,s,ld", [(5000, 4, 300, 5003), (3 * 4096 + 17, 3, 512, 3 * 4096 + 18)])
def test_hrht_strided_columns(api, m, n, s, ld):
    # leading dimension above m (odd: the 16-byte load path is off)
    rng = np.random.default_rng(m + ld)
    A = rng.standard_normal((m, n))
    buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    buf[:, :m] = torch.as_tensor(A.T.copy(), device="cuda")
    d = api.desc(api.NS_HRHT, s=s, seed=2)
    got = api.ns_sketch(d, buf.t()[:m, :]).cpu().numpy()
    ref = O.hrht(2, s, A)
    for c in range(n):
        assert np.max(np.abs(got[:, c] - ref[:, c])) <= 2.0 ** -40 * np.max(np.abs(ref[:, c]))


def test_hrht_solve_exact_null_space(api):
    # Algorithm 1 with the H-RHT on an exact 4-dimensional null space
    w = workloads.at_scale(seed=4, m=1 << 14, n=64, null_dim=4)
    A = w["A"]
    d = api.desc(api.NS_HRHT, s=256, seed=3)
    Vk, sk, _, status = api.ns_solve(d, api.colmajor(A, device="cuda"), 4, save=False)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Vk = Vk.cpu().numpy()
    ref = O.solve(O.HRHT, 3, 256, A, 4)
    assert sine(ref["Vk"], Vk) < 1e-8
    assert sine(w["V"][:, -4:], Vk) < 1e-9
    assert O.residual(A, Vk) <= 1e-12 * np.linalg.norm(A)


def test_hrht_wide_dynamic_range_and_zero_column(api):
    # columns from 1e-200 to 1e200, a column of zeros, and one large entry in
    # an otherwise tiny column (its block sets the column quantum)
    rng = np.random.default_rng(2)
    m, n, s = 20000, 5, 256
    A = rng.standard_normal((m, n))
    A[:, 0] *= 1e-200
    A[:, 1] *= 1e200
    A[:, 2] = 0.0
    A[:, 3] *= 1e-6
    A[12345, 3] = 1e6
    got = sketch(api, A, s, 6)
    ref = O.hrht(6, s, A)
    assert np.all(got[:, 2] == 0.0)
    for c in (0, 1, 3, 4):
        assert np.max(np.abs(got[:, c] - ref[:, c])) <= 2.0 ** -40 * np.max(np.abs(ref[:, c]))


def test_hrht_exact_null_vector_gpu(api):
    # m' = 4^8, so the 1/sqrt(m') scale is a power of two and SA stays exact
    rng = np.random.default_rng(5)
    m, n = 60000, 6
    B = rng.integers(-20, 21, size=(m, n - 1)).astype(np.float64)
    z = rng.integers(-3, 4, size=n - 1).astype(np.float64)
    A = np.column_stack([B, B @ z])
    x = np.concatenate([z, [-1.0]])
    SA = sketch(api, A, 512, 3)
    assert np.all(SA @ x == 0)


def test_hrht_repeatable(api):
    rng = np.random.default_rng(8)
    A = rng.standard_normal((1 << 16, 6))
    a = sketch(api, A, 700, 1)
    b = sketch(api, A, 700, 1)
    assert np.array_equal(a, b)


def test_hrht_nonfinite_flag(api):
    A = np.ones((9000, 3))
    A[4321, 1] = np.inf
    d = api.desc(api.NS_HRHT, s=64, seed=0)
    Vk, sk, _, status = api.ns_solve(d, api.colmajor(A, device="cuda"), 1, save=False)
    torch.cuda.synchronize()
    assert int(status.item()) == api._lib.NS_ERR_NONFINITE


def test_hrht_solve_coherent_example(api):
    # Figure 1's difficult example (U = [I_n; 0], m = 1000, n = 100, s = 2n):
    # the SRHT fails, the H-RHT returns the null vector within Theorem 3.2.
    m, n, s = 1000, 100, 200
    U = np.zeros((m, n))
    U[:n, :n] = np.eye(n)
    V = workloads.orthonormal(np.random.default_rng(3), n, n)
    sig = np.concatenate([np.ones(n - 2), [0.1, 1e-6]])
    A = np.asfortranarray(workloads.from_svd(U, sig, V))
    out = {}
    for kind in (api.NS_SRHT, api.NS_HRHT):
        d = api.desc(kind, s=s, seed=1)
        Vk, sk, _, status = api.ns_solve(d, api.colmajor(A, device="cuda"), 1, save=False)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        out[kind] = (Vk.cpu().numpy(), sk.cpu().numpy())
    assert sine(V[:, -1:], out[api.NS_SRHT][0]) > 0.5
    ref = O.solve(O.HRHT, 1, s, A, 1)
    Vh, sh = out[api.NS_HRHT]
    assert sine(ref["Vk"], Vh) < 1e-8
    R = np.linalg.qr(O.hrht(1, s, U), mode="r")
    bound = np.linalg.norm(R - np.linalg.inv(R).T, 2) / chi(sh[0] ** 2, sig[n - 2] ** 2)
    assert sine(V[:, -1:], Vh) <= bound * (1 + 1e-6) < 1e-4


@pytest.mark.slow
def test_hrht_at_scale_sampled_columns(api):
    # the benchmark's workload (m = 2^20, n = 256, s = 1024) sketched in one
    # launch; four columns checked against the oracle one by one
    w = workloads.at_scale(seed=0)
    A = w["A"]
    got = sketch(api, A, 1024, 0)
    for c in (0, 97, 200, 255):
        ref = O.hrht(0, 1024, A[:, c:c + 1])[:, 0]
        assert np.max(np.abs(got[:, c] - ref)) <= 2.0 ** -40 * np.max(np.abs(ref))
