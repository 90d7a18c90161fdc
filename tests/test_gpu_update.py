"""Section 5 row updates of a sketch through ns_sketch_update against the
oracle's sketch_update: the regenerated SRHT and sparse-sign columns are exact
(+-1/sqrt(s), +-1/sqrt(zeta)), the Gaussian column is FP64 Box-Muller on both
sides, so the results agree to a few units of rounding of ||SA||."""
import numpy as np
import pytest

import oracle as O

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


KINDS = {"srht": O.SRHT, "sparse": O.SPARSE_SIGN, "gauss": O.GAUSSIAN}


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("op,j", [(1, 0), (1, 4097), (1, 5000 - 1), (0, 5000), (0, 5123), (1, 5050)])
def test_row_update_parity(api, kind, op, j):
    rng = np.random.default_rng(len(kind) * 100 + j)
    m0, n, s = 5000, 7, 96
    SA = np.asfortranarray(rng.standard_normal((s, n)))
    row = rng.standard_normal(n)
    k = KINDS[kind]
    kd = {"srht": api.NS_SRHT, "sparse": api.NS_SPARSE_SIGN, "gauss": api.NS_GAUSSIAN}[kind]
    d = api.desc(kd, s=s, seed=9, zeta=8)
    SAd = api.colmajor(SA, device="cuda")
    api.ns_sketch_update(d, m0, op, j, torch.as_tensor(row, device="cuda"), SAd)
    torch.cuda.synchronize()
    ref = O.sketch_update(k, 9, s, SA, m0, op, j, row, zeta=8)
    np.testing.assert_allclose(SAd.cpu().numpy(), ref, rtol=0, atol=1e-14 * np.linalg.norm(ref))


def test_row_remove_matches_resketch(api):
    # ns_sketch of A, then removing row j, equals ns_sketch of A with row j zeroed
    rng = np.random.default_rng(5)
    m, n, s, j = 10000, 6, 128, 7777
    A = np.asfortranarray(rng.standard_normal((m, n)))
    d = api.desc(api.NS_SRHT, s=s, seed=4)
    SA = api.ns_sketch(d, api.colmajor(A, device="cuda"))
    api.ns_sketch_update(d, m, api.NS_ROW_REMOVE, j, torch.as_tensor(A[j, :].copy(), device="cuda"), SA)
    A0 = A.copy(order="F")
    A0[j, :] = 0.0
    ref = api.ns_sketch(d, api.colmajor(A0, device="cuda"))
    torch.cuda.synchronize()
    np.testing.assert_allclose(SA.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=1e-12 * np.linalg.norm(A))
