"""GPU parity of the sparse-sign sketch against the oracle.

Bit-exact: the (row, sign) realisation of every column of S, and SA on
integer inputs (the GPU sums are exact integers scaled once by 1/sqrt(zeta)).
FP64 inputs: |SA - SA_oracle| <= 1e-12 ||A||_F entrywise.
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


def dev(api, A):
    return api.colmajor(np.asfortranarray(A), device="cuda")


@pytest.mark.parametrize("m,s,zeta,seed", [(1, 1, 1, 0), (1000, 50, 8, 3), (4097, 1024, 8, 0), (777, 300, 13, 5),
                                           ((1 << 20), 1024, 8, 1)])
def test_sparse_meta_bitexact(api, m, s, zeta, seed):
    d = api.desc(api.NS_SPARSE_SIGN, s=s, seed=seed, zeta=zeta)
    rows, signs = api.ns_sparse_meta(d, m)
    r_or, g_or = O.sparse_sign_cols(seed, s, zeta, m)
    assert np.array_equal(rows.cpu().numpy(), r_or)
    assert np.array_equal(signs.cpu().numpy(), g_or)


# s <= 1024 with zeta <= 8 takes the gather form (target-sorted 512-row chunks,
# register accumulators, 16 columns per CTA); larger s or zeta the scatter form.
# The gather cases include ragged row and column counts, several chunk ranges
# per column group, and the three register-tile sizes (s <= 256, 512, 1024).
SHAPES = [(1, 1, 1, 1), (100, 3, 16, 4), (1000, 33, 300, 8), (5000, 64, 256, 8), (9999, 17, 1000, 8),
          ((1 << 16) + 3, 40, 512, 8), ((1 << 18), 2, 2048, 8), (3000, 5, 70, 13),
          ((1 << 17) + 333, 17, 1024, 8), (70001, 33, 513, 8), (40000, 5, 257, 4), (511, 16, 64, 8)]


@pytest.mark.parametrize("m,n,s,zeta", SHAPES)
def test_sparse_sketch_parity(api, m, n, s, zeta):
    rng = np.random.default_rng(m + 7 * n)
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-3, 3, size=(1, n)))
    d = api.desc(api.NS_SPARSE_SIGN, s=s, seed=2, zeta=zeta)
    SA = api.ns_sketch(d, dev(api, A)).cpu().numpy()
    ref = O.sparse_sign(2, s, zeta, A)
    assert np.max(np.abs(SA - ref)) <= 1e-12 * np.linalg.norm(A)


def test_sparse_odd_leading_dimension(api):
    # lda odd: the staged copies fall back from 16-byte to 8-byte pieces
    rng = np.random.default_rng(41)
    m, n, s, ld = 20001, 19, 512, 20003
    A = rng.standard_normal((m, n))
    buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    buf[:, :m] = torch.as_tensor(A.T.copy(), device="cuda")
    d = api.desc(api.NS_SPARSE_SIGN, s=s, seed=6, zeta=8)
    SA = api.ns_sketch(d, buf.t()[:m, :]).cpu().numpy()
    assert np.max(np.abs(SA - O.sparse_sign(6, s, 8, A))) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("m,n,s", [(3000, 7, 128), ((1 << 15) + 11, 3, 1024), (50000, 21, 600)])
def test_sparse_integer_inputs_bitexact(api, m, n, s):
    rng = np.random.default_rng(m)
    A = rng.integers(-1000, 1001, size=(m, n)).astype(np.float64)
    d = api.desc(api.NS_SPARSE_SIGN, s=s, seed=9, zeta=8)
    SA = api.ns_sketch(d, dev(api, A)).cpu().numpy()
    assert np.array_equal(SA, O.sparse_sign(9, s, 8, A, scaled=False) * (1.0 / np.sqrt(8.0)))


def test_sparse_solve_parity(api):
    w = workloads.graded(seed=5, m=20000, n=48, k=3, tail=1e-9)
    A = w["A"]
    d = api.desc(api.NS_SPARSE_SIGN, s=192, seed=4, zeta=8)
    Vk, sk, _, status = api.ns_solve(d, dev(api, A), 3)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = O.solve(O.SPARSE_SIGN, 4, 192, A, 3, zeta=8)
    Vg = Vk.cpu().numpy()
    n = A.shape[1]
    assert O.residual(A, Vg) <= (1 + 1e-10) * O.residual(A, ref["Vk"]) + 10 * 2.0 ** -53 * np.sqrt(n) * np.linalg.norm(A)
    assert sine(ref["Vk"], Vg) < 1e-8


@pytest.mark.slow
def test_sparse_at_scale_full_size(api):
    # the benchmark workload with the sparse-sign sketch (zeta = 8, s = 1024)
    w = workloads.at_scale(seed=0)
    A = w["A"]
    d = api.desc(api.NS_SPARSE_SIGN, s=1024, seed=0, zeta=8)
    Ad = dev(api, A)
    SA = api.ns_sketch(d, Ad).cpu().numpy()
    cols = [0, 77, 255]
    ref = O.sparse_sign(0, 1024, 8, A[:, cols])
    assert np.max(np.abs(SA[:, cols] - ref)) <= 1e-12 * np.linalg.norm(A)
    Vk, sk, _, status = api.ns_solve(d, Ad, 4)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert sine(w["V"][:, -4:], Vk.cpu().numpy()) < 1e-9
