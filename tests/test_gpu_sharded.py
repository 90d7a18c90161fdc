"""ns_sketch_rows: the share S[:, o:o+m_p] A_p of a row block in the sketch of
the whole A, against ns_sketch and the oracle.

The shares of blocks that cover every row must add up to the sketch: the SRHT
transforms each block's 4096-row pieces with their global indices (signs of D,
row parities of H), and the sparse sign's column j belongs to global row j.
Blocks are cut on 4096-row boundaries (as the multi-GPU driver cuts them) and
also at arbitrary rows (a block boundary inside a 4096-row piece: both sides
read the other's rows as zero).  Tolerance: each share is a sum of FP64 chunk
partials, so the sum of shares differs from the sketch by the rounding of those
sums, ~u ||A||_F: asserted at 1e-12 ||A||_F (and 8 u max|SA| on integer data,
where every partial is exact and only the 1/sqrt(s) scaling rounds).
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_00975_gb300 import sharded

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


def sum_of_shares(api, d, Ad, cuts):
    m = Ad.shape[0]
    total = None
    for o, e in zip(cuts[:-1], cuts[1:]):
        part = api.ns_sketch_rows(d, Ad[o:e], o, m)
        total = part.clone() if total is None else total + part
    torch.cuda.synchronize()
    return total


@pytest.mark.parametrize("kind", ["SRHT", "SPARSE_SIGN"])
@pytest.mark.parametrize("m,n,s,cuts", [
    (4 * 4096, 3, 128, "aligned4"), (3 * 4096 + 777, 5, 256, "aligned2"), (50000, 4, 512, [0, 1, 4095, 9000, 50000]),
    (3000, 2, 64, [0, 1234, 3000]), ((1 << 17) + 3, 6, 1024, "aligned3")])
def test_shares_add_up_to_the_sketch(api, kind, m, n, s, cuts):
    rng = np.random.default_rng(m + n)
    d = api.desc(getattr(api, "NS_" + kind), s=s, seed=5, zeta=8)
    if isinstance(cuts, str):
        parts = sharded.row_partition(m, int(cuts[-1]))
        cuts = [o for o, _ in parts] + [m]
    for integer in (False, True):
        A = rng.integers(-20, 21, size=(m, n)).astype(np.float64) if integer else rng.standard_normal((m, n))
        Ad = api.colmajor(A, device="cuda")
        got = sum_of_shares(api, d, Ad, cuts).cpu().numpy()
        ref = api.ns_sketch(d, Ad).cpu().numpy()
        if integer:
            assert np.max(np.abs(got - ref)) <= 8 * U53 * np.max(np.abs(ref))
        else:
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.linalg.norm(A)
        orc = O.sketch(0 if kind == "SRHT" else 1, 5, s, A, zeta=8)
        assert np.max(np.abs(got - orc)) <= 1e-12 * np.linalg.norm(A)


def test_shares_at_benchmark_size(api):
    # the benchmark's A (2^20 x 256) cut into four 2^18-row blocks, as four GPUs
    # would hold it
    m, n, s = 1 << 20, 256, 1024
    g = torch.Generator(device="cuda").manual_seed(2)
    Ad = torch.randn((n, m), generator=g, device="cuda", dtype=torch.float64).t()
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    cuts = [o for o, _ in sharded.row_partition(m, 4)] + [m]
    got = sum_of_shares(api, d, Ad, cuts)
    ref = api.ns_sketch(d, Ad)
    assert float((got - ref).abs().max()) <= 1e-12 * float(torch.linalg.norm(Ad))


def test_sketch_rows_rejects_bad_blocks(api):
    A = api.colmajor(np.ones((100, 3)), device="cuda")
    d = api.desc(api.NS_SRHT, s=32, seed=0)
    with pytest.raises(api.NSError):
        api.ns_sketch_rows(d, A, 50, 120)      # rows 50..149 beyond m_total = 120
    with pytest.raises(api.NSError):
        api.ns_sketch_rows(api.desc(api.NS_HRHT, s=32, seed=0), A, 0, 100)   # H-RHT: not offered
