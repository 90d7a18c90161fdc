"""GPU adjoint (ns_backward and the autograd.Function) against the oracle,
central finite differences of the GPU forward, and the full-size workload.

Loss: L = ||W W^T Z||_F^2 (invariant under W -> W Q), dL/dW = 2 Z Z^T W.
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_00975_gb300 import workloads

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


def loss_grad(Vk, Z):
    P = Vk @ Vk.T
    return float(np.linalg.norm(P @ Z) ** 2), 2.0 * Z @ Z.T @ Vk


def problem(m, n, k, seed):
    rng = np.random.default_rng(seed)
    U = workloads.orthonormal(rng, m, n)
    V = workloads.orthonormal(rng, n, n)
    sig = np.concatenate([np.linspace(3, 1, n - k), np.logspace(-3, -4, k)])
    return workloads.from_svd(U, sig, V), rng.standard_normal((n, 4))


@pytest.mark.parametrize("m,n,k,s", [(5000, 12, 3, 48), (4096, 33, 1, 132), (70001, 20, 4, 80)])
def test_backward_matches_oracle(api, m, n, k, s):
    A, Z = problem(m, n, k, m + n)
    d = api.desc(api.NS_SRHT, s=s, seed=3)
    Ad = api.colmajor(A, device="cuda")
    Vk, sk, sv, status = api.ns_solve(d, Ad, k)
    Vg = Vk.cpu().numpy()
    _, dV = loss_grad(Vg, Z)
    dA = api.ns_backward(d, m, n, k, sv, Vk, api.colmajor(dV, device="cuda")).cpu().numpy()
    SA, V, sigma = [x.cpu().numpy() for x in api.unpack_save(sv, s, n)]
    ref = O.backward_srht(3, s, m, SA, V, sigma, Vg, dV)
    assert np.linalg.norm(dA - ref) <= 1e-10 * np.linalg.norm(ref)


def test_backward_finite_differences_gpu(api):
    m, n, k, s = 6000, 10, 2, 40
    A, Z = problem(m, n, k, 11)
    d = api.desc(api.NS_SRHT, s=s, seed=5)

    def fwd(Ah):
        Vk, _, sv, _ = api.ns_solve(d, api.colmajor(Ah, device="cuda"), k)
        return Vk, sv

    Vk, sv = fwd(A)
    _, dV = loss_grad(Vk.cpu().numpy(), Z)
    dA = api.ns_backward(d, m, n, k, sv, Vk, api.colmajor(dV, device="cuda")).cpu().numpy()
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(3):
        E = rng.standard_normal((m, n))
        Lp = loss_grad(fwd(A + h * E)[0].cpu().numpy(), Z)[0]
        Lm = loss_grad(fwd(A - h * E)[0].cpu().numpy(), Z)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(float(np.sum(dA * E)) - fd) <= 1e-6 * abs(fd) + 1e-9


def test_autograd_function(api):
    from paper_2206_00975_gb300.autograd import null_space
    m, n, k, s = 3000, 9, 2, 36
    A, Z = problem(m, n, k, 4)
    At = api.colmajor(A, device="cuda").requires_grad_(True)
    Zt = torch.as_tensor(Z, device="cuda")
    W, sk = null_space(At, k, s, seed=7)
    L = torch.linalg.norm(W @ (W.T @ Zt)) ** 2
    L.backward()
    out = O.solve(O.SRHT, 7, s, A, k)
    _, dV = loss_grad(out["Vk"], Z)
    ref = O.backward_srht(7, s, m, out["SA"], out["V"], out["sigma"], out["Vk"], dV)
    assert np.linalg.norm(At.grad.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_backward_rejects_bad_k(api):
    d = api.desc(api.NS_SRHT, s=16, seed=0)
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(api.NSError):
        api.ns_backward(d, 100, 4, 4, x, x, x, dA=api._empty_cm(100, 4, "cuda"))


@pytest.mark.slow
def test_backward_adjoint_workload_full_size(api):
    # m = 2^18, n = 128, k = 8, s = 512, Z ~ N(0,1)^{128 x 16}
    w = workloads.adjoint(seed=0)
    A, Z = w["A"], w["W"]
    m, n = A.shape
    k, s = 8, 512
    d = api.desc(api.NS_SRHT, s=s, seed=0)
    Vk, sk, sv, status = api.ns_solve(d, api.colmajor(A, device="cuda"), k)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Vg = Vk.cpu().numpy()
    _, dV = loss_grad(Vg, Z)
    dA = api.ns_backward(d, m, n, k, sv, Vk, api.colmajor(dV, device="cuda")).cpu().numpy()
    SA, V, sigma = [x.cpu().numpy() for x in api.unpack_save(sv, s, n)]
    ref = O.backward_srht(0, s, m, SA, V, sigma, Vg, dV)
    assert np.linalg.norm(dA - ref) <= 1e-10 * np.linalg.norm(ref)
