"""GPU parity of the SRHT sketch and Algorithm 1 against the oracle.

Tolerances (stated by the scope of this library):
  * signs and sample rows: bit-exact;
  * SA in FP64: |SA - SA_oracle| <= 1e-12 ||A||_F entrywise (integer inputs:
    bit-exact, since the fixed-point path is exact on them);
  * solve: ||A V||_F <= (1 + 1e-10) ||A V_oracle||_F + 10 u sqrt(n) ||A||_F, and
    the subspace sine <= 1e-8 whenever u sigma_1 / gap <= 1e-10 (else reported).
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


def to_dev(api, A, ld=None):
    A = np.asfortranarray(A)
    m, n = A.shape
    if ld is None or ld == m:
        return api.colmajor(A, device="cuda")
    buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    buf[:, :m] = torch.as_tensor(A.T.copy(), device="cuda")
    return buf.t()[:m, :]


def words_to_signs(words, length):
    w = words.cpu().numpy().astype(np.uint32)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little")[:length]
    return np.where(bits == 1, -1, 1).astype(np.int8)


@pytest.mark.parametrize("m,s,seed", [(1, 1, 0), (37, 16, 1), (4096, 128, 0), (5000, 512, 7), (1 << 20, 1024, 3)])
def test_srht_meta_bitexact(api, m, s, seed):
    d = api.desc(api.NS_SRHT, s=s, seed=seed)
    words, rows = api.ns_srht_meta(d, m)
    lg = O.ceil_log2(m)
    assert np.array_equal(words_to_signs(words, 1 << lg), O.signs(seed, 1 << lg))
    assert np.array_equal(rows.cpu().numpy().astype(np.int64), O.sample_rows(seed, lg, s))


SHAPES = [
    (1, 1, 1, None), (37, 3, 16, None), (64, 5, 64, 67), (4096, 7, 128, None), (5000, 4, 256, 5003),
    (3 * 4096 + 17, 3, 512, 3 * 4096 + 18), ((1 << 16) + 5, 2, 1024, None), (1 << 18, 3, 2048, None),
]


@pytest.mark.parametrize("m,n,s,ld", SHAPES)
def test_srht_sketch_parity(api, m, n, s, ld):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-3, 3, size=(1, n)))
    d = api.desc(api.NS_SRHT, s=s, seed=5)
    SA = api.ns_sketch(d, to_dev(api, A, ld)).cpu().numpy()
    ref = O.srht(5, s, A)
    err = np.max(np.abs(SA - ref))
    assert err <= 1e-12 * np.linalg.norm(A), (err, np.linalg.norm(A))


@pytest.mark.parametrize("m,n,s", [(300, 6, 64), (9000, 3, 256), ((1 << 15) + 1, 2, 512)])
def test_srht_integer_inputs_bitexact(api, m, n, s):
    rng = np.random.default_rng(m)
    A = rng.integers(-1000, 1001, size=(m, n)).astype(np.float64)
    d = api.desc(api.NS_SRHT, s=s, seed=11)
    SA = api.ns_sketch(d, to_dev(api, A)).cpu().numpy()
    assert np.array_equal(SA, O.srht(11, s, A))


@pytest.mark.parametrize("m,n,s", [((1 << 20) - 3, 128, 1000), (1 << 20, 130, 1024), ((1 << 19) + 4097, 64, 1025),
                                   ((1 << 18) + 1, 40, 100), (20000, 3, 16384)])
def test_srht_sketch_sampled_columns(api, m, n, s):
    # chunked geometries (up to 16 blocks per fixed-point accumulator, ragged
    # last block) and the largest s the library takes (its sampled sums fill
    # most of a CTA's shared memory) compared with the oracle on a few columns;
    # the sketch acts on each column alone
    g = torch.Generator(device="cuda")
    g.manual_seed(m + n + s)
    A = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g).t()
    A = A * torch.exp(torch.linspace(-3.0, 3.0, n, dtype=torch.float64, device="cuda"))[None, :]
    d = api.desc(api.NS_SRHT, s=s, seed=8)
    SA = api.ns_sketch(d, A).cpu().numpy()
    cols = [0, n // 2, n - 1]
    Ah = A[:, cols].cpu().numpy()
    ref = O.srht(8, s, Ah)
    assert np.max(np.abs(SA[:, cols] - ref)) <= 1e-12 * np.linalg.norm(Ah)


@pytest.mark.parametrize("m,n,s", [(1 << 12, 3, 64), (1 << 16, 5, 1000), (1 << 18, 9, 1024), (1 << 19, 4, 3000),
                                   (1 << 20, 256, 1024)])
def test_srht_block_forms_agree_bitwise(api, m, n, s):
    # ns_sketch (256-thread block pipeline) and the whole-window share of
    # ns_sketch_rows (128-thread block pipeline) quantise the same chunks the
    # same way and add exactly, so for m a power of two (the same chunking)
    # they agree bit for bit, up to the benchmark's size
    g = torch.Generator(device="cuda")
    g.manual_seed(m + s)
    A = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=g).t()
    A = A * torch.exp(torch.linspace(-20.0, 20.0, n, dtype=torch.float64, device="cuda"))[None, :]
    d = api.desc(api.NS_SRHT, s=s, seed=4)
    a = api.ns_sketch(d, A)
    b = api.ns_sketch_rows(d, A, 0, m)
    assert torch.equal(a, b)


def test_srht_wide_dynamic_range(api):
    # entries spanning 1e-200..1e+200 in one column: error bound is relative to ||A||_F
    rng = np.random.default_rng(3)
    m, n, s = 20000, 2, 256
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-200, 200, size=(m, n))
    d = api.desc(api.NS_SRHT, s=s, seed=2)
    SA = api.ns_sketch(d, to_dev(api, A)).cpu().numpy()
    ref = O.srht(2, s, A)
    assert np.max(np.abs(SA - ref)) <= 1e-12 * np.linalg.norm(A)


def test_srht_tiny_and_subnormal_entries(api):
    # columns whose largest entry lies below 2^(P - 1023) (about 1e-294) take
    # the quantiser's exact-subnormal path; subnormal entries are mixed in.
    # Norms are taken on scaled copies (squares of 1e-309 underflow).
    rng = np.random.default_rng(12)
    m, n, s = 20000, 3, 256
    A = rng.standard_normal((m, n)) * 1e-300
    A[::7, 1] = 5e-324 * rng.integers(-1000, 1001, size=A[::7, 1].shape)
    A[:, 2] *= 1e-9
    d = api.desc(api.NS_SRHT, s=s, seed=6)
    SA = api.ns_sketch(d, to_dev(api, A)).cpu().numpy()
    ref = O.srht(6, s, A)
    for c in range(n):
        nrm = np.linalg.norm(A[:, c] * 2.0 ** 1000) * 2.0 ** -1000
        assert nrm > 0
        assert np.max(np.abs(SA[:, c] - ref[:, c])) <= 1e-12 * nrm, c


def test_srht_exact_null_vector_gpu(api):
    rng = np.random.default_rng(2)
    m, n = 6000, 6
    B = rng.integers(-20, 21, size=(m, n - 1)).astype(np.float64)
    z = rng.integers(-3, 4, size=n - 1).astype(np.float64)
    A = np.column_stack([B, B @ z])
    d = api.desc(api.NS_SRHT, s=64, seed=4)
    SA = api.ns_sketch(d, to_dev(api, A)).cpu().numpy() * 8.0   # sqrt(64) = 8: integers again
    assert np.all(SA @ np.concatenate([z, [-1.0]]) == 0)


def test_srht_nonfinite_flag(api):
    A = np.ones((5000, 2))
    A[123, 1] = np.nan
    d = api.desc(api.NS_SRHT, s=32, seed=0)
    Ad = to_dev(api, A)
    Vk, sk, sv, status = api.ns_solve(d, Ad, 1)
    torch.cuda.synchronize()
    assert int(status.item()) == api._lib.NS_ERR_NONFINITE


# ------------------------------------------------------------------ solve ----
def check_solve(A, Vk, sk, ref, sigma_full_ref):
    n = A.shape[1]
    normA = np.linalg.norm(A)
    r_gpu = O.residual(A, Vk)
    r_or = O.residual(A, ref["Vk"])
    assert r_gpu <= (1 + 1e-10) * r_or + 10 * U53 * np.sqrt(n) * normA, (r_gpu, r_or)
    k = Vk.shape[1]
    sig = np.sort(sigma_full_ref)[::-1]
    gap = sig[n - k - 1] - sig[n - k] if k < n else np.inf
    s_val = sine(ref["Vk"], Vk) if k < n else 0.0
    if U53 * sig[0] / gap <= 1e-10:
        assert s_val <= 1e-8, s_val
    np.testing.assert_allclose(sk, ref["sigk"], rtol=1e-6, atol=20 * U53 * np.sqrt(n) * sig[0])
    return s_val


def run_solve(api, A, s, k, seed):
    d = api.desc(api.NS_SRHT, s=s, seed=seed)
    Vk, sk, sv, status = api.ns_solve(d, to_dev(api, A), k)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return Vk.cpu().numpy(), sk.cpu().numpy(), sv


def test_solve_plain_workload(api):
    w = workloads.plain(seed=0)
    Vk, sk, sv = run_solve(api, w["A"], w["s"], w["k"], 0)
    ref = O.solve(O.SRHT, 0, w["s"], w["A"], w["k"])
    check_solve(w["A"], Vk, sk, ref, ref["sigma"])
    # against the true null vector: a-priori bound of Section 3.1.1
    assert sine(w["V"][:, -1:], Vk) < 1e-7


@pytest.mark.parametrize("m,n,k,s", [(3000, 24, 2, 96), (2048, 1, 1, 1), (513, 8, 8, 8), (777, 17, 3, 34),
                                     (20000, 64, 5, 256)])
def test_solve_shapes(api, m, n, k, s):
    w = workloads.graded(seed=m + n, m=m, n=n, k=min(k, n), tail=1e-9) if n > 1 else None
    A = w["A"] if w else np.random.default_rng(0).standard_normal((m, n))
    Vk, sk, _ = run_solve(api, A, s, k, 9)
    ref = O.solve(O.SRHT, 9, s, A, k)
    check_solve(A, Vk, sk, ref, ref["sigma"])


def test_solve_exact_null_space(api):
    rng = np.random.default_rng(6)
    m, n, k = 4096, 24, 3
    B = rng.standard_normal((m, n - k))
    Z = rng.standard_normal((n - k, k))
    A = np.asfortranarray(np.column_stack([B, B @ Z]))
    Vk, sk, _ = run_solve(api, A, 96, k, 1)
    assert sine(np.vstack([Z, -np.eye(k)]), Vk) < 1e-12
    assert O.residual(A, Vk) < 1e-13 * np.linalg.norm(A)


def test_solve_save_buffer(api):
    w = workloads.graded(seed=4, m=5000, n=16, k=2)
    s = 64
    d = api.desc(api.NS_SRHT, s=s, seed=3)
    Vk, sk, sv, status = api.ns_solve(d, to_dev(api, w["A"]), 2)
    SA, V, sigma = api.unpack_save(sv, s, 16)
    ref = O.solve(O.SRHT, 3, s, w["A"], 2)
    assert np.max(np.abs(SA.cpu().numpy() - ref["SA"])) <= 1e-12 * np.linalg.norm(w["A"])
    Vn = V.cpu().numpy()
    assert np.linalg.norm(Vn.T @ Vn - np.eye(16)) < 1e-13
    np.testing.assert_allclose(np.sort(sigma.cpu().numpy())[::-1], np.sort(ref["sigma"])[::-1], rtol=1e-9,
                               atol=1e-15)


@pytest.mark.slow
def test_solve_at_scale_full_size(api):
    # the benchmark's workload: m = 2^20, n = 256, k = 4 exact null space, SRHT s = 1024
    w = workloads.at_scale(seed=0)
    A = w["A"]
    Vk, sk, _ = run_solve(api, A, 1024, 4, 0)
    ref = O.solve(O.SRHT, 0, 1024, A, 4)
    check_solve(A, Vk, sk, ref, ref["sigma"])
    assert sine(w["V"][:, -4:], Vk) < 1e-9


def test_residual_gpu(api):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((70000, 12))
    W = rng.standard_normal((12, 3))
    got = float(api.ns_residual(to_dev(api, A), api.colmajor(W, device="cuda")).item())
    assert abs(got - np.linalg.norm(A @ W)) <= 1e-12 * np.linalg.norm(A @ W)


# ------------------------------------------------------------- FP32 stream ----
@pytest.mark.parametrize("m,n,s", [(4096, 3, 128), (5000, 4, 256), (9000, 3, 700), ((1 << 18) + 3, 2, 2048),
                                   (8197, 2, 2100)])
def test_srht_fp32_stream_parity(api, m, n, s):
    # s <= 2048 keeps the sampled rows' sums in registers; larger s in shared memory
    # FP32 arithmetic: error bound u32 * (log2 m' + 2) * ||A||_F per entry
    rng = np.random.default_rng(m)
    A32 = rng.standard_normal((m, n)).astype(np.float32)
    d = api.desc(api.NS_SRHT, s=s, seed=4, prec=api.NS_PREC_FP32_STREAM)
    SA = api.ns_sketch(d, api.colmajor(A32, device="cuda")).cpu().numpy()
    A64 = A32.astype(np.float64)
    ref = O.srht(4, s, A64)
    tol = 2.0 ** -24 * (O.ceil_log2(m) + 2) * np.linalg.norm(A64)
    assert np.max(np.abs(SA - ref)) <= tol


def test_solve_fp32_stream_reports_error(api):
    w = workloads.graded(seed=2, m=1 << 14, n=32, k=2, tail=1e-9, dtype=np.float32)
    A32 = w["A"]
    A64 = A32.astype(np.float64)
    d = api.desc(api.NS_SRHT, s=128, seed=1, prec=api.NS_PREC_FP32_STREAM)
    Vk, sk, _, status = api.ns_solve(d, api.colmajor(A32, device="cuda"), 2)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = O.solve(O.SRHT, 1, 128, A64, 2)
    r_gpu, r_or = O.residual(A64, Vk.cpu().numpy()), O.residual(A64, ref["Vk"])
    # FP32 sketch noise ~ u32 ||A||: the residual stays within that of the FP64 oracle's
    assert r_gpu <= r_or + 2.0 ** -24 * 20 * np.linalg.norm(A64)
