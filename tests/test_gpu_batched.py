"""GPU parity of ns_solve_batched (uneven TLS and general problems) against the
oracle, per problem, and against single-problem ns_solve.

TLS (Section 4): x = -v(1:n)/v(n+1) from the trailing right singular vector of
the sketched [X b]; compared with the oracle's sketched TLS on the same sketch
(relative 1e-8, the gap sigma_n(X)/sigma_{n+1}([X b]) ~ 1e3 allows it).
"""
import numpy as np
import pytest

import oracle as O
from paper_2206_00975_gb300 import workloads
from tests.helpers import sine

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


def test_batched_tls_matches_oracle(api):
    ms, ns = workloads.tls_batch_shapes(seed=3, batch=24, m_lo=2048, m_hi=20000, n_lo=8, n_hi=64)
    rng = np.random.default_rng(5)
    probs, host = [], []
    for i, (m, n) in enumerate(zip(ms, ns)):
        Xb, x_true = workloads.tls_problem(rng, int(m), int(n))
        s = 2 * (int(n) + 1)
        host.append((Xb, s, 100 + i))
        probs.append({"A": api.colmajor(Xb, device="cuda"), "s": s, "k": 1, "seed": 100 + i, "tls": True})
    outs, status, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for (Xb, s, seed), (Vk, sk, x) in zip(host, outs):
        x_or, v_or, st = O.tls(seed, s, Xb)
        assert st == O.OK
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - x_or) <= 1e-8 * np.linalg.norm(x_or)
        assert sine(v_or[:, None], Vk.cpu().numpy()) < 1e-8


def test_batched_tls_benchmark_shapes(api):
    # a seeded subset of the batched workload's 4096 shapes (m uniform in
    # [2^11, 2^16], n uniform in [8, 128]), with its largest-n and largest-m
    # problems, all in one persistent launch, against the oracle per problem
    ms, ns = workloads.tls_batch_shapes(seed=0, batch=4096)
    pick = sorted(set(np.random.default_rng(8).choice(4096, 14, replace=False).tolist() +
                      [int(np.argmax(ns)), int(np.argmax(ms))]))
    rng = np.random.default_rng(13)
    probs, host = [], []
    for i in pick:
        m, n = int(ms[i]), int(ns[i])
        Xb, _ = workloads.tls_problem(rng, m, n)
        s = 2 * (n + 1)
        host.append((Xb, s, i))
        probs.append({"A": api.colmajor(Xb, device="cuda"), "s": s, "k": 1, "seed": i, "tls": True})
    assert max(p["A"].shape[1] for p in probs) == 129 and max(p["A"].shape[0] for p in probs) >= 65000
    outs, status, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for (Xb, s, seed), (Vk, sk, x) in zip(host, outs):
        x_or, v_or, st = O.tls(seed, s, Xb)
        assert st == O.OK
        v = Vk.cpu().numpy()[:, 0]
        # the gap sigma_n(X) / sigma_{n+1}([X b]) of these problems is ~1e2..1e3 at
        # s = 2(n + 1): the TLS solution is determined to ~u * 1e3 relative
        assert np.linalg.norm(x.cpu().numpy() - x_or) <= 1e-8 * np.linalg.norm(x_or)
        assert sine(v_or[:, None], v[:, None]) < 1e-8
        r_gpu, r_or = O.residual(Xb, v[:, None]), O.residual(Xb, v_or[:, None])
        assert r_gpu <= (1 + 1e-10) * r_or + 10 * U53 * np.sqrt(Xb.shape[1]) * np.linalg.norm(Xb)


def test_batched_fp32_stream_matches_oracle(api):
    # FP32-stored [X b] through the FP32-stream sketch (FP32 butterflies and
    # accumulation; QR and Jacobi in FP64), against the oracle's FP64 solve of
    # the same FP32 data: the sketch noise (~2^-24 ||A|| per entry) is far below
    # the TLS noise level (1e-3), so the residual matches the oracle's and x
    # agrees to ~1e-4 relative
    ms, ns = workloads.tls_batch_shapes(seed=7, batch=12, m_lo=2048, m_hi=40000, n_lo=8, n_hi=100)
    rng = np.random.default_rng(17)
    probs, host = [], []
    for i, (m, n) in enumerate(zip(ms, ns)):
        Xb, _ = workloads.tls_problem(rng, int(m), int(n))
        Xb32 = Xb.astype(np.float32)
        s = 2 * (int(n) + 1)
        host.append((Xb32.astype(np.float64), s, 300 + i))
        probs.append({"A": api.colmajor(Xb32, device="cuda"), "s": s, "k": 1, "seed": 300 + i, "tls": True})
    outs, status, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for (Xb, s, seed), (Vk, sk, x) in zip(host, outs):
        x_or, v_or, st = O.tls(seed, s, Xb)
        assert st == O.OK
        v = Vk.cpu().numpy()
        r_gpu, r_or = O.residual(Xb, v), O.residual(Xb, v_or[:, None])
        assert r_gpu <= r_or * (1 + 1e-3)
        assert np.linalg.norm(x.cpu().numpy() - x_or) <= 1e-4 * np.linalg.norm(x_or)


def test_batched_tuning_keeps_the_bits(api):
    # the launch knobs (panel width, persistent grid sizes) change the work
    # distribution only: every setting gives the default's results bit for bit
    ms, ns = workloads.tls_batch_shapes(seed=9, batch=40, m_lo=2048, m_hi=30000, n_lo=8, n_hi=90)
    rng = np.random.default_rng(3)
    probs = []
    for i, (m, n) in enumerate(zip(ms, ns)):
        Xb, _ = workloads.tls_problem(rng, int(m), int(n))
        A = api.colmajor(Xb if i % 2 else Xb.astype(np.float32), device="cuda")   # FP64 and FP32 problems mixed
        probs.append({"A": A, "s": 2 * (int(n) + 1), "k": 1, "seed": i, "tls": True})
    ref, st0, _ = api.ns_solve_batched(probs, tuning={})
    torch.cuda.synchronize()
    ref = [[t.clone() for t in o] for o in ref]
    for setting in ({"panel": 2}, {"panel": 4, "sketch_ctas_per_sm": 2}, {"panel": 3, "dense_ctas_per_sm": 1},
                    {"panel": 1, "sketch_ctas_per_sm": 1, "dense_ctas_per_sm": 2}):
        outs, st, _ = api.ns_solve_batched(probs, tuning=setting)
        torch.cuda.synchronize()
        assert torch.equal(st, st0)
        for o, r in zip(outs, ref):
            for a, b in zip(o, r):
                assert torch.equal(a, b), setting
    api.ns_solve_batched(probs[:1], tuning={})   # back to the defaults


def test_autotuner_caches_a_setting_with_the_same_bits(api, tmp_path):
    from paper_2206_00975_gb300 import autotune
    ms, ns = workloads.tls_batch_shapes(seed=4, batch=48, m_lo=2048, m_hi=20000, n_lo=8, n_hi=64)
    rng = np.random.default_rng(8)
    probs = []
    for i, (m, n) in enumerate(zip(ms, ns)):
        Xb, _ = workloads.tls_problem(rng, int(m), int(n))
        probs.append({"A": api.colmajor(Xb, device="cuda"), "s": 2 * (int(n) + 1), "k": 1, "seed": i, "tls": True})
    path = str(tmp_path / "tuning.json")
    ref, _, _ = api.ns_solve_batched(probs, tuning={})
    torch.cuda.synchronize()
    ref = [[t.clone() for t in o] for o in ref]
    (outs, st, keep), setting = autotune.solve_batched_tuned(probs, cache_path=path)
    torch.cuda.synchronize()
    assert autotune.lookup(probs, cache_path=path) == setting
    for o, r in zip(outs, ref):
        for a, b in zip(o, r):
            assert torch.equal(a, b)
    api.ns_solve_batched(probs[:1], tuning={})


def test_batched_general_problems(api):
    rng = np.random.default_rng(9)
    shapes = [(5000, 24, 96, 2), (300, 3, 8, 1), (4096, 32, 128, 4), (9000, 17, 40, 17), (70000, 40, 200, 3)]
    probs, refs = [], []
    for i, (m, n, s, k) in enumerate(shapes):
        w = workloads.graded(seed=i, m=m, n=n, k=min(k, n), tail=1e-9)
        probs.append({"A": api.colmajor(w["A"], device="cuda"), "s": s, "k": k, "seed": 7 * i + 1})
        refs.append((w["A"], O.solve(O.SRHT, 7 * i + 1, s, w["A"], k)))
    outs, status, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    for (A, ref), (Vk, sk, _) in zip(refs, outs):
        Vg = Vk.cpu().numpy()
        n = A.shape[1]
        r_gpu, r_or = O.residual(A, Vg), O.residual(A, ref["Vk"])
        assert r_gpu <= (1 + 1e-10) * r_or + 10 * U53 * np.sqrt(n) * np.linalg.norm(A)
        if Vg.shape[1] < n:
            assert sine(ref["Vk"], Vg) < 1e-8
        np.testing.assert_allclose(sk.cpu().numpy(), ref["sigk"], rtol=1e-6, atol=1e-14)


def test_batched_matches_single_solves(api):
    rng = np.random.default_rng(2)
    probs, singles = [], []
    for i in range(6):
        m, n = int(rng.integers(3000, 9000)), int(rng.integers(5, 30))
        A = np.asfortranarray(rng.standard_normal((m, n)))
        Ad = api.colmajor(A, device="cuda")
        probs.append({"A": Ad, "s": 2 * n, "k": 2, "seed": i})
        d = api.desc(api.NS_SRHT, s=2 * n, seed=i)
        Vk, sk, _, _ = api.ns_solve(d, Ad, 2)
        singles.append((Vk.cpu().numpy(), sk.cpu().numpy()))
    outs, status, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    for (Vk, sk, _), (V1, s1) in zip(outs, singles):
        np.testing.assert_allclose(sk.cpu().numpy(), s1, rtol=1e-12)
        assert sine(V1, Vk.cpu().numpy()) < 1e-10


def test_batched_per_problem_status(api):
    rng = np.random.default_rng(1)
    A1 = rng.standard_normal((2000, 6))
    A2 = A1.copy()
    A2[17, 3] = np.inf
    X = rng.standard_normal((3000, 4))
    X[:, 3] = X[:, 2]
    Xb = np.column_stack([X, rng.standard_normal(3000)])  # null vector e3 - e4: no TLS solution
    probs = [{"A": api.colmajor(A1, device="cuda"), "s": 12, "k": 1, "seed": 1},
             {"A": api.colmajor(A2, device="cuda"), "s": 12, "k": 1, "seed": 1},
             {"A": api.colmajor(Xb, device="cuda"), "s": 10, "k": 1, "seed": 2, "tls": True}]
    outs, status, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert st[0] == 0
    assert st[1] == api._lib.NS_ERR_NONFINITE
    assert st[2] == api._lib.NS_ERR_TLS_NOSOLUTION


def test_batched_rejects_invalid_problem(api):
    A = api.colmajor(np.ones((100, 4)), device="cuda")
    with pytest.raises(api.NSError):
        api.ns_solve_batched([{"A": A, "s": 2, "k": 1, "seed": 0}])      # s < n
    with pytest.raises(api.NSError):
        api.ns_solve_batched([{"A": A, "s": 8, "k": 2, "seed": 0, "tls": True}])  # TLS needs k = 1
