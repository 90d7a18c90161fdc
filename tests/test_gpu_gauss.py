"""GPU Gaussian sketch on the tensor cores (3-term BF16 split, FP32 accumulation)
against the oracle's FP64 Gaussian sketch.

Error model: each operand x is split into hi + lo with |x - hi - lo| <= 2^-18
|x|; the three kept products miss about 3 * 2^-18 of |g a| each; G itself is
generated in FP32 (relative ~1e-6 against the oracle's FP64 Box-Muller) and
the tiles accumulate in FP32.  The entrywise bound used is
|SA - SA_oracle| <= 2^-12 * sqrt(sum_j (g_rj a_jc)^2 * m) / sqrt(s) in the
root-mean-square sense, checked as a relative Frobenius error of 1e-4 per
column plus an absolute floor.
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


@pytest.mark.parametrize("m,n,s", [(1000, 16, 128), (5000, 37, 200), (3001, 300, 256), (20000, 512, 128),
                                   (64, 3, 16), (1 << 16, 64, 384)])
def test_gaussian_sketch_parity(api, m, n, s):
    rng = np.random.default_rng(m + n)
    A32 = rng.standard_normal((m, n)).astype(np.float32)
    SA = gauss_gpu(api, A32, s, 7)
    cols = list(range(n)) if n <= 40 else sorted(set([0, 1, n // 2, n - 2, n - 1]))
    ref = O.gaussian(7, s, A32.astype(np.float64), cols=cols)
    for c in cols:
        err = np.linalg.norm(SA[:, c] - ref[:, c])
        assert err <= 1e-4 * np.linalg.norm(ref[:, c]) + 1e-12, (c, err, np.linalg.norm(ref[:, c]))


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
