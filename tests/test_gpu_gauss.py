"""GPU Gaussian sketch on the tensor cores (3-term BF16 split, FP32 accumulation)
against the oracle's FP64 Gaussian sketch, entry by entry.

Error model of one entry SA[r, c] = sum_j T_j / sqrt(s), T_j = g_rj a_jc,
with mag = sqrt(sum_j T_j^2) / sqrt(s) the size of its terms (computed by the
oracle):

* Split.  Each operand x is split as hi = bf16(x) (|x - hi| <= 2^-8 |x|) and
  lo = bf16(x - hi) (|x - hi - lo| <= 2^-16 |x|); the three kept products
  hi hi + hi lo + lo hi miss lo lo and the two split residuals, at most
  3 * 2^-16 |T_j| per term, with signs that vary from term to term, so their
  sum is a random walk: a few times 2^-17 mag.  (G itself is generated in FP32,
  a relative ~2^-20 per entry: smaller.)
* Accumulation.  Each CTA accumulates one split of K = kper rows of A in FP32
  in tensor memory, 16 rows per step and three products per step.  If every
  such addition loses up to one unit in the last place of the running sum
  S_k (2^-23 |S_k|, alignment without rounding), the losses add up to
  3 * 2^-23 sum_k |S_k|; S_k is a random walk of step 4 sigma_T
  (sigma_T = mag sqrt(s / m) / sqrt(s) per term), so the expected sum is
  sqrt(2/pi) 4 (2/3) (kper/16)^(3/2) sigma_T.  The nsplit splits are summed
  in FP64.  This term grows like m at fixed s: measured on the GPU, the median
  of |err| / mag went 5e-6, 1.8e-5, 6.8e-5 for m = 2^14, 2^16, 2^18 at s = 2048,
  n = 512, which is the scaling of this model (a random-walk rounding error
  would grow like sqrt(m)).

The bound asserted per entry is
  mag * (2^-13 + 2 * 3 * 2^-23 * E(kper) * sqrt(nsplit) / sqrt(m)),
E(K) = sqrt(2/pi) 4 (2/3) (K/16)^(3/2): the split part at ~8 standard
deviations and twice the expected accumulation loss.
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


def split_geometry(m, s):
    """(kper, nsplit) of the tensor-core sketch: one CTA per (128-row tile of
    SA, split of the rows of A), about one CTA per SM, splits in 32-row steps."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mtiles = -(-s // 128)
    nsplit = max(sms // mtiles, 1)
    kchunks = -(-m // 32)
    nsplit = min(nsplit, kchunks)
    kper = -(-kchunks // nsplit) * 32
    return kper, -(-m // kper)


def entry_tol(m, s):
    kper, nsplit = split_geometry(m, s)
    e_sum = np.sqrt(2 / np.pi) * 4 * (2 / 3) * (kper / 16) ** 1.5
    return 2.0 ** -13 + 2 * 3 * 2.0 ** -23 * e_sum * np.sqrt(nsplit) / np.sqrt(m)


def check_rows(SA, A64, s, seed, rows):
    m = A64.shape[0]
    ref, mag = O.gaussian_rows(seed, s, A64, rows)
    err = np.abs(SA[rows] - ref)
    tol = entry_tol(m, s)
    worst = float(np.max(err / np.maximum(mag, 1e-300)))
    assert np.all(err <= tol * mag + 1e-300), (worst, tol)
    return worst, tol


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
    worst, tol = check_rows(SA, A32.astype(np.float64), s, 11, rows)
    print("gaussian s=2048 n=512 m=2^18: worst |err| / mag = %.3e (bound %.3e)" % (worst, tol))


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
