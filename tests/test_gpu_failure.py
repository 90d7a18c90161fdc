"""Failure detection on the GPU without a fault or a hang.

* Every spin wait in the kernels is bounded.  ns_test_bounded_wait makes two of
  them run out on purpose (the grid barrier of the cooperative kernels and the
  cluster-peer mbarrier wait of the ring Jacobi): each must write
  NS_ERR_TIMEOUT and return promptly, and the stream must stay usable.
* A Jacobi sweep limit the iteration reaches (the descriptor's max_sweeps)
  must give NS_ERR_NOCONV with the partial result written: finite singular
  values and orthonormal V.
* Reads of unwritten scratch: every solve is run once with a zero-filled and
  once with a NaN-filled (all bytes 0xFF) workspace; the results must be
  identical bit for bit.
"""
import ctypes
import time

import numpy as np
import pytest

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


def _small_sketch_ok(api):
    A = api.colmajor(np.random.default_rng(0).standard_normal((3000, 5)), device="cuda")
    SA = api.ns_sketch(api.desc(api.NS_SRHT, s=64, seed=1), A)
    torch.cuda.synchronize()
    return bool(torch.isfinite(SA).all().item())


@pytest.mark.parametrize("which,limit", [(0, 1000), (1, 20000)])
def test_bounded_wait_times_out(api, which, limit):
    lib = api._lib.load()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = lib.ns_test_bounded_wait(which, limit, ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                  ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert int(status.item()) == api._lib.NS_ERR_TIMEOUT
    assert _small_sketch_ok(api)  # the context and the stream are still usable


@pytest.mark.parametrize("sketched", [False, True])
def test_sweep_limit_reports_noconv_with_partial_result(api, sketched):
    w = workloads.graded(seed=4, m=1 << 13, n=48, k=2)
    A = api.colmajor(w["A"], device="cuda")
    d = api.desc(api.NS_SRHT, s=4 * 48, seed=2, max_sweeps=1)
    if sketched:
        SA = api.ns_sketch(d, A)
        Vk, sk, sv, status = api.ns_solve_sketched(d, SA, 2, save=True)
    else:
        Vk, sk, sv, status = api.ns_solve(d, A, 2, save=True)
    torch.cuda.synchronize()
    assert int(status.item()) == api._lib.NS_ERR_NOCONV
    _, V, sigma = api.unpack_save(sv, d.s, 48)
    V = V.cpu().numpy()
    assert np.isfinite(sigma.cpu().numpy()).all() and np.isfinite(Vk.cpu().numpy()).all()
    assert np.linalg.norm(V.T @ V - np.eye(48)) < 1e-12
    # the default limit converges on the same input
    d0 = api.desc(api.NS_SRHT, s=4 * 48, seed=2)
    _, _, _, st0 = api.ns_solve(d0, A, 2, save=True)
    torch.cuda.synchronize()
    assert int(st0.item()) == 0


def _poison(ws, nan):
    ws.fill_(255 if nan else 0)
    return ws


def _twice(fn):
    """fn(nan) -> list of tensors; returns both runs on host."""
    outs = []
    for nan in (False, True):
        r = fn(nan)
        torch.cuda.synchronize()
        outs.append([t.cpu().clone() for t in r])
    return outs


@pytest.mark.parametrize("kind,prec,dtype,s", [
    ("SRHT", "PREC_FP64", np.float64, 256), ("SPARSE_SIGN", "PREC_FP64", np.float64, 256),
    ("HRHT", "PREC_FP64", np.float64, 256), ("SRHT", "PREC_FP32_STREAM", np.float32, 256),
    ("GAUSSIAN", "PREC_BF16X3", np.float32, 256)])
def test_solve_ignores_workspace_contents(api, kind, prec, dtype, s):
    w = workloads.graded(seed=9, m=(1 << 15) + 77, n=64, k=2)
    A = api.colmajor(w["A"].astype(dtype), device="cuda")
    d = api.desc(getattr(api, "NS_" + kind), s=s, seed=3, prec=getattr(api, "NS_" + prec))
    ws = api.workspace(d, A.shape[0], 64, 2, "cuda")

    def run(nan):
        Vk, sk, sv, st = api.ns_solve(d, A, 2, save=True, ws=_poison(ws, nan))
        return [Vk, sk, sv, st]
    a, b = _twice(run)
    assert int(a[3].item()) == 0
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_other_entry_points_ignore_workspace_contents(api):
    rng = np.random.default_rng(5)
    m, n, k, s = 20000, 24, 3, 96
    A = api.colmajor(rng.standard_normal((m, n)), device="cuda")
    d = api.desc(api.NS_SRHT, s=s, seed=7)
    ws = api.workspace(d, m, n, k, "cuda")
    SA = api.ns_sketch(d, A)
    Vk, sk, sv, _ = api.ns_solve(d, A, k, save=True)
    dV = api.colmajor(rng.standard_normal((n, k)), device="cuda")

    def run(nan):
        out = list(api.ns_solve_sketched(d, SA, k, save=True, ws=_poison(ws, nan)))
        Ve, se, ke, sve, ste = api.ns_solve_eps(d, A, 0.5, save=True, ws=_poison(ws, nan))
        kk = int(ke.item())   # columns past k of Ve (entries past k of se) are not written
        out += [Ve[:, :kk], se[:kk], ke, sve, ste]
        out.append(api.ns_backward(d, m, n, k, sv, Vk, dV, ws=_poison(ws, nan)))
        return out
    a, b = _twice(run)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_batched_ignores_workspace_contents(api):
    rng = np.random.default_rng(6)
    probs = []
    for i, (mi, ni) in enumerate([(3000, 9), (5000, 17), (2100, 33)]):
        Xb, _ = workloads.tls_problem(rng, mi, ni)
        probs.append({"A": api.colmajor(Xb, device="cuda"), "s": 2 * (ni + 1), "k": 1, "seed": i, "tls": True})
    outs0, st0, keep0 = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    ws = keep0[2]

    def run(nan):
        outs, st, keep = api.ns_solve_batched(probs, ws=_poison(ws, nan))
        return [t for o in outs for t in o] + [st]
    a, b = _twice(run)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
