"""The tolerance version of Algorithm 1 (Section 2, after Algorithm 1) through
ns_solve_eps, against the oracle's: the same count k = #{sigma_i < eps} (the
inputs keep every singular value far from eps, so rounding cannot move one
across it), the same subspace, singular values to 1e-12 sigma_1."""
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


def run(api, A, s, eps, seed=0):
    d = api.desc(api.NS_SRHT, s=s, seed=seed)
    Vk, sk, kt, _, status = api.ns_solve_eps(d, api.colmajor(np.asfortranarray(A), device="cuda"), eps, save=False)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    k = int(kt.item())
    return Vk[:, :k].cpu().numpy(), sk[:k].cpu().numpy(), k


@pytest.mark.parametrize("m,n,null_dim", [(2048, 24, 3), (1 << 14, 64, 4), (4096, 256, 4)])
def test_eps_exact_null_space(api, m, n, null_dim):
    w = workloads.at_scale(seed=m + n, m=m, n=n, null_dim=null_dim)
    A, s = w["A"], 4 * n
    eps = 1e-10 * np.linalg.norm(A, 2)
    Vg, sg, k = run(api, A, s, eps)
    Vo, so, ko, full = O.solve_eps(O.SRHT, 0, s, A, eps)
    assert k == ko == null_dim
    assert sine(Vo, Vg) < 1e-8
    assert np.max(np.abs(sg - so)) <= 1e-12 * full["sigma"].max()
    assert np.linalg.norm(A @ Vg) <= 1e-12 * np.linalg.norm(A)


def test_eps_plain_workload(api):
    # sigma_32 = 1e-12 against sigma_31 = 1e-4: eps = 1e-8 takes the last one only
    w = workloads.plain(seed=0)
    Vg, sg, k = run(api, w["A"], w["s"], 1e-8)
    Vo, so, ko, _ = O.solve_eps(O.SRHT, 0, w["s"], w["A"], 1e-8)
    assert k == ko == 1
    assert sine(Vo, Vg) < 1e-8


def test_eps_limits(api):
    w = workloads.plain(seed=2, m=512, n=12)
    _, _, k0 = run(api, w["A"], 48, 0.0)
    assert k0 == 0
    Vg, sg, kn = run(api, w["A"], 48, 4.0 * np.linalg.norm(w["A"], 2))
    assert kn == 12
    assert np.all(np.diff(sg) <= 0)
    np.testing.assert_allclose(Vg.T @ Vg, np.eye(12), atol=1e-13)


# (The GPU Gaussian sketch is BF16x3 on FP32 input, ~1e-7 accurate: its
# Theorem 3.4 case is pinned on the oracle only.)
@pytest.mark.parametrize("kind", [O.SRHT, O.SPARSE_SIGN])
def test_larger_subspace_theorem_3_4(api, kind):
    # Theorem 3.4: A's trailing k = 4 singular values are 1e-2 .. 1e-3 with no
    # gap among them. The GPU's trailing k sketched vectors contain A's
    # trailing l = 2 (case 2), and its trailing l lie in A's trailing k
    # (case 1), within the theorem's bounds on the realized S; the k-space
    # matches the oracle's (gap tilde sigma_{n-k} / tilde sigma_{n-k+1} ~ 100).
    rng = np.random.default_rng(50 + kind)
    m, n, s, k, l = 1000, 100, 400, 4, 2
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.ones(n - k), np.logspace(-2, -3, k)])
    A = workloads.from_svd(U, sig, V)
    gkind = {O.SRHT: api.NS_SRHT, O.SPARSE_SIGN: api.NS_SPARSE_SIGN}[kind]
    d = api.desc(gkind, s=s, seed=23)
    Vk, sk, _, status = api.ns_solve(d, api.colmajor(A, device="cuda"), k, save=False)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Vk, sk = Vk.cpu().numpy(), sk.cpu().numpy()
    out = O.solve(kind, 23, s, A, k)
    st = np.sort(out["sigma"])[::-1]
    assert sine(out["Vk"], Vk) < 1e-8
    np.testing.assert_allclose(sk, out["sigk"], rtol=1e-9)
    R = np.linalg.qr(O.sketch(kind, 23, s, U), mode="r")
    Mnorm = np.linalg.norm(R - np.linalg.inv(R).T, 2)
    b1 = Mnorm / chi(st[n - l] ** 2, sig[n - k - 1] ** 2)
    b2 = Mnorm / chi(sig[n - l] ** 2, st[n - k - 1] ** 2)
    assert max(b1, b2) < 0.05
    assert sine(V[:, n - k:], Vk[:, k - l:]) <= b1 * (1 + 1e-6)
    assert sine(Vk, V[:, n - l:]) <= b2 * (1 + 1e-6)
