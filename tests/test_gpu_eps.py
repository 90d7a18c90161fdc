"""The tolerance version of Algorithm 1 (Section 2, after Algorithm 1) through
ns_solve_eps, against the oracle's: the same count k = #{sigma_i < eps} (the
inputs keep every singular value far from eps, so rounding cannot move one
across it), the same subspace, singular values to 1e-12 sigma_1."""
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
