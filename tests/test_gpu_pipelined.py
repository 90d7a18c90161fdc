"""ns_solve_pipelined: a stream of problems, the sketch of problem i + 1
running while the dense stage of problem i is past its QRs, gives for every
problem ns_solve's result bit for bit (the same kernels in the same order
per problem), whatever the overlap."""
import numpy as np
import pytest

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


def rank_deficient(rng, m, n, k):
    # A = G1 G2 with G1 m x (n - k), G2 (n - k) x n: a k-dimensional null space
    return rng.standard_normal((m, n - k)) @ rng.standard_normal((n - k, n))


@pytest.mark.parametrize("kind,m,n,s,k,count", [
    ("srht", 1 << 15, 256, 1024, 4, 7),    # both QRs fused, FP32 phase, completions; every lane twice
    ("srht", 20000, 96, 384, 3, 4),        # ragged m, n < 128
    ("sparse", 1 << 14, 64, 256, 2, 3),
    ("srht", 5000, 40, 160, 1, 2),         # no FP32 phase (n < 64)
    ("hrht", 1 << 14, 64, 256, 2, 4),
    ("gauss", 8192, 64, 256, 2, 4),        # FP32-stored A, BF16x3 tensor-core sketch
    ("srht", 4096, 32, 128, 1, 1),         # a single problem
])
def test_pipelined_matches_ns_solve(api, kind, m, n, s, k, count):
    rng = np.random.default_rng(m + n + count)
    dtype = torch.float32 if kind == "gauss" else torch.float64
    As = [api.colmajor(rank_deficient(rng, m, n, k), dtype=dtype, device="cuda") for _ in range(count)]
    if kind == "srht":
        d = api.desc(api.NS_SRHT, s=s, seed=3)
    elif kind == "hrht":
        d = api.desc(api.NS_HRHT, s=s, seed=3)
    elif kind == "gauss":
        d = api.desc(api.NS_GAUSSIAN, s=s, seed=3, prec=api.NS_PREC_BF16X3)
    else:
        d = api.desc(api.NS_SPARSE_SIGN, s=s, seed=3, zeta=8)
    Vks, sig, status = api.ns_solve_pipelined(d, As, k)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * count
    for i, A in enumerate(As):
        Vk, sk, _, st = api.ns_solve(d, A, k, save=False)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert torch.equal(Vks[i], Vk), i
        assert torch.equal(sig[i], sk), i


def test_pipelined_on_a_side_stream_orders_with_it(api):
    # work enqueued on the caller's stream before the call is seen by it, and
    # work enqueued after it sees the results
    rng = np.random.default_rng(5)
    m, n, s, k = 8192, 64, 256, 2
    d = api.desc(api.NS_SRHT, s=s, seed=1)
    src = [api.colmajor(rank_deficient(rng, m, n, k), device="cuda") for _ in range(2)]
    As = [torch.zeros_like(a) for a in src]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for a, b in zip(As, src):
            a.copy_(b)
        Vks, sig, status = api.ns_solve_pipelined(d, As, k, stream=side)
        out = torch.stack([v.clone() for v in Vks])
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, 0]
    for i in range(2):
        Vk, sk, _, _ = api.ns_solve(d, src[i], k, save=False)
        torch.cuda.synchronize()
        assert torch.equal(out[i], Vk)
