"""GPU AAA with a reused SRHT sketch (Section 6.2) against the oracle.

AAA is greedy: rounding can flip a near-tie of the argmax, so parity is
checked teacher-forced: the oracle replays the GPU's support points and both
sides must agree on the incrementally updated sketch (a row downdate and a
column update per iteration, against a fresh sketch of the final Loewner
matrix), on the weights and on the error trajectory.
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


def run_gpu(api, x, f, K, smax, seed, forced=None, sketch=False):
    xd = torch.as_tensor(x, device="cuda")
    fd = torch.as_tensor(f, device="cuda")
    fo = None if forced is None else torch.as_tensor(np.asarray(forced, dtype=np.int64), device="cuda")
    out = api.ns_aaa_real(xd, fd, K, smax, seed=seed, forced=fo, want_sketch=sketch)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) and k != "_ws" else v) for k, v in out.items()}


def test_aaa_teacher_forced_parity(api):
    x, f = workloads.aaa_points(seed=1, m=1 << 14, scale=50.0)
    K, smax, seed = 40, 160, 3
    g = run_gpu(api, x, f, K, smax, seed, sketch=True)
    assert g["status"][0] == 0
    assert len(set(g["support"].tolist())) == K
    sup, W, err, st, SAk = O.aaa(seed, x, f, K, smax, forced=g["support"], return_sketch=True)
    # the incrementally updated sketch equals the oracle's (same support sequence)
    assert np.max(np.abs(g["SAk"] - SAk)) <= 1e-11 * np.max(np.abs(SAk))
    # ... and a fresh sketch of the final Loewner matrix (support rows zeroed)
    L = np.zeros((x.size, K))
    for l, jl in enumerate(g["support"]):
        with np.errstate(divide="ignore", invalid="ignore"):
            L[:, l] = (f - f[jl]) / (x - x[jl])
    L[g["support"], :] = 0.0
    assert np.max(np.abs(g["SAk"] - O.srht(seed, smax, L))) <= 1e-11 * np.max(np.abs(SAk))
    # error trajectory: equal (to 5% in log) until convergence; once either
    # side is at rounding level (below 1e-9) the other must be too
    for k in range(K):
        eg, eo = g["errmax"][k], err[k]
        if min(eg, eo) > 1e-9:
            assert abs(np.log10(eg) - np.log10(eo)) < 0.05, (k, eg, eo)
        else:
            assert max(eg, eo) < 1e-8, (k, eg, eo)
    for k in range(1, 12):   # early iterations are well separated
        assert sine(W[k - 1, :k, None], g["W"][k - 1, :k, None]) < 1e-8


def test_aaa_converges_free_running(api):
    x, f = workloads.aaa_points(seed=0, m=1 << 15, scale=50.0)
    g = run_gpu(api, x, f, 60, 240, 1)
    assert g["errmax"][-1] < 1e-10 * np.abs(f).max()
    sup_or, _, err_or, _ = O.aaa(1, x, f, 60, 240)
    # free-running trajectories agree to within a few iterations of convergence
    k_gpu = int(np.argmax(g["errmax"] < 1e-9))
    k_or = int(np.argmax(err_or < 1e-9))
    assert abs(k_gpu - k_or) <= 3


def test_aaa_graph_capture_replays_identically(api):
    x, f = workloads.aaa_points(seed=2, m=1 << 13, scale=30.0)
    K, smax = 20, 80
    xd = torch.as_tensor(x, device="cuda")
    fd = torch.as_tensor(f, device="cuda")
    eager = api.ns_aaa_real(xd, fd, K, smax, seed=4)
    torch.cuda.synchronize()
    ws = eager["_ws"]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.ns_aaa_real(xd, fd, K, smax, seed=4, ws=ws, stream=s)   # warm-up on the capture stream
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        out = api.ns_aaa_real(xd, fd, K, smax, seed=4, ws=ws, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out["support"], eager["support"])
    assert torch.equal(out["W"], eager["W"])
    assert torch.equal(out["errmax"], eager["errmax"])


@pytest.mark.slow
def test_aaa_full_size_workload(api):
    # 2^17 points in [-1, 1], f = tanh(50 x), 100 iterations, s = 4k prefix of a 400-row sketch
    x, f = workloads.aaa_points(seed=0, m=1 << 17, scale=50.0)
    g = run_gpu(api, x, f, 100, 400, 0, sketch=True)
    assert g["status"][0] == 0
    sup, W, err, st, SAk = O.aaa(0, x, f, 100, 400, forced=g["support"], return_sketch=True)
    assert np.max(np.abs(g["SAk"] - SAk)) <= 1e-10 * np.max(np.abs(SAk))
    # AAA converges (to ~1e-13 here, near iteration 25) and then keeps adding
    # support points to an ever worse conditioned Loewner matrix: past that
    # point the error is set by rounding, for the oracle replaying the same
    # support points as much as for the GPU (both wander between 1e-11 and
    # 1e-7).  So: the GPU converges, and its error after the last iteration is
    # no worse than the oracle's on the same support points.
    fmax = np.abs(f).max()
    assert g["errmax"].min() < 1e-12 * fmax
    assert g["errmax"][-1] <= max(1e-10 * fmax, 10.0 * err[-1])
