"""GPU Gaussian sketch on the tensor cores (3-term BF16 split, FP32 accumulation)
against the oracle's FP64 Gaussian sketch, entry by entry.

Error model of one entry SA[r, c] = sum_j g_rj a_jc / sqrt(s).  Each operand
x is split as hi = bf16(x) (|x - hi| <= 2^-8 |x|) and lo = bf16(x - hi)
(|x - hi - lo| <= 2^-16 |x|); the three kept products hi hi + hi lo + lo hi
miss lo lo and the two split residuals, at most 3 * 2^-16 |g a| per term,
with signs that vary from term to term.  G is generated in FP32 (the oracle
evaluates Box-Muller in FP64), a relative ~2^-20 per entry, and the split-K
partials accumulate in FP32 (2^-24 per addition of a running sum).  The terms'
errors add like a random walk, so the error of the entry is a small multiple
of 2^-17 * mag with mag = sqrt(sum_j (g_rj a_jc)^2) / sqrt(s), the size of its
terms (computed by the oracle).  The bound asserted per entry is
2^-12 * mag: about 6 standard deviations over the entries checked.
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_00975_gb300 import workloads
from tests.helpers import sine

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


def gauss_gpu(api, A32, s, seed):
    d = api.desc(api.NS_GAUSSIAN, s=s, seed=seed, prec=api.NS_PREC_BF16X3)
    return api.ns_sketch(d, api.colmajor(A32, device="cuda")).cpu().numpy()


ENTRY_TOL = 2.0 ** -12


def check_rows(SA, A64, s, seed, rows):
    ref, mag = O.gaussian_rows(seed, s, A64, rows)
    err = np.abs(SA[rows] - ref)
    worst = float(np.max(err / np.maximum(mag, 1e-300)))
    assert np.all(err <= ENTRY_TOL * mag + 1e-300), worst
    return worst


@pytest.mark.parametrize("m,n,s", [(1000, 16, 128), (5000, 37, 200), (3001, 300, 256), (20000, 512, 128),
                                   (64, 3, 16), (1 << 16, 64, 384)])
def test_gaussian_sketch_parity(api, m, n, s):
    rng = np.random.default_rng(m + n)
    A32 = rng.standard_normal((m, n)).astype(np.float32)
    SA = gauss_gpu(api, A32, s, 7)
    rows = list(range(s)) if s * m * n <= (1 << 27) else sorted(set(rng.integers(0, s, 24).tolist() + [0, s - 1]))
    check_rows(SA, A32.astype(np.float64), s, 7, rows)


def test_gaussian_sketch_parity_precision_geometry(api):
    # the precision workload's sketch geometry: s = 2048 (16 row tiles of 128),
    # n = 512 (the full TMEM width), and m = 2^18, split over several K ranges;
    # rows sampled from every row tile (the oracle forms each row in O(m n))
    m, n, s = 1 << 18, 512, 2048
    rng = np.random.default_rng(31)
    A32 = rng.standard_normal((m, n)).astype(np.float32)
    SA = gauss_gpu(api, A32, s, 11)
    rows = sorted(set([128 * t + int(rng.integers(0, 128)) for t in range(16)] + [0, 1, s - 1]))
    worst = check_rows(SA, A32.astype(np.float64), s, 11, rows)
    print("gaussian s=2048 n=512 m=2^18: worst |err| / mag = %.3e (bound %.3e)" % (worst, ENTRY_TOL))


def test_gaussian_is_deterministic_and_seeded(api):
    rng = np.random.default_rng(1)
    A32 = rng.standard_normal((4000, 24)).astype(np.float32)
    a = gauss_gpu(api, A32, 96, 3)
    b = gauss_gpu(api, A32, 96, 3)
    c = gauss_gpu(api, A32, 96, 4)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)


def test_gaussian_solve(api):
    # a trailing pair well separated from the rest (gap 0.1 against the
    # ~1e-5 split-product error), so the sketched subspace is resolved
    rng = np.random.default_rng(3)
    m, n = 1 << 14, 40
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.logspace(0, -1, n - 2), [1e-3, 1e-3]])
    A32 = workloads.from_svd(U, sig, V).astype(np.float32)
    A64 = A32.astype(np.float64)
    d = api.desc(api.NS_GAUSSIAN, s=160, seed=5, prec=api.NS_PREC_BF16X3)
    Vk, sk, _, status = api.ns_solve(d, api.colmajor(A32, device="cuda"), 2)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = O.solve(O.GAUSSIAN, 5, 160, A64, 2)
    Vg = Vk.cpu().numpy()
    # the split-product error (~1e-5 of ||A||) perturbs the sketch: residual and
    # subspace stay within that level of the FP64 oracle's
    assert O.residual(A64, Vg) <= O.residual(A64, ref["Vk"]) + 1e-4 * np.linalg.norm(A64)
    assert sine(ref["Vk"], Vg) < 1e-3
    assert sine(V[:, -2:], Vg) < 1e-1
