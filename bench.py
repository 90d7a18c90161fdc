#!/usr/bin/env python
"""Benchmark of the sketch-and-solve null-space hot path (Algorithm 1) on GB300.

Headline workload (one step = one full solve): A = U diag(sigma) V^T with
m = 2^20, n = 256, sigma_1..252 log-spaced from 1 to 1e-6 and a 4-dimensional
exact null space; SRHT sketch with s = 1024; FP64 QR of the sketch, QR of R^T,
FP32 linear phase and FP64 one-sided Jacobi SVD; the k = 4 trailing right
singular vectors.  A (2 GiB) is larger than L2, so every step streams it from
HBM.  The same workload is also solved with the sparse-sign sketch (zeta = 8)
and the H-RHT.  The other workloads (plain, precision, adjoint, batched TLS
and AAA) are timed in the same run, each with its own recipe, and reported
under "configs".

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
    python bench.py --case NAME      # one kernel family on a small case (profiling)

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own replica of the workload (weak scaling; the path needs no collective).
"""
import argparse
import concurrent.futures
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, S, K_NULL, SEED = 1 << 20, 256, 1024, 4, 0
E2E_PARTS = 4   # concurrent host-to-device copies per step in the end-to-end leg
# DRAM bytes of one srht_f64_chunk256_kernel launch at full size: dram__bytes_read.sum
# + dram__bytes_write.sum of the ncu capture at m = 2^19, n = 64 (268.64 MB read +
# 3.12 MB written), scaled by the 8x the full launch processes
SRHT_TRAFFIC = (268.64e6 + 3.12e6) * 8
SRHT_TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum at m=2^19 n=64, scaled x8"
METRIC = "null-space solves/s and sketch HBM GB/s (% of peak) at stated ||AV||_F accuracy"
WORKLOAD = "at_scale: m=2^20 n=256 FP64 column-major, sigma log-spaced 1..1e-6 + 4 exact zeros, SRHT s=1024, k=4"
FP64_FLOPS_PER_CLK_SM = 4.0   # 2 FP64 FMA per clock per SM (bench.py --case fp64peak measures the rate)


def bench_config(world):
    """The config dict both arms print (identical keys and values)."""
    return {"workload": WORKLOAD, "l2": "input larger than L2 (2 GiB A per step)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops", 1906.5)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(seed):
    from paper_2206_00975_gb300 import workloads
    return workloads.at_scale(seed=seed, m=M, n=N, null_dim=K_NULL)


def dense_flops(s, n, k, stats):
    """Algorithmic FP64 flops of lines 3-4 of Algorithm 1 as the GPU runs them:
    Householder QR of s x n, Householder QR of n x n, one-sided Jacobi (dot
    products 6n per visited pair, rotation of two columns of X and of V 12n),
    the n^3 products after the FP32 phase (when it ran): V0 made orthogonal
    (two symmetric products, n^3 each, and one 2n^3) and applied to X0 and Q2
    (2n^3 each), then two first-order completions (G = X^T X and K^2, n^3
    each, K^4 and K^6 when formed, n^3 each, and X Q, V Q, 2n^3 each), and
    the k trailing columns of V (4 n^2 k).  The FP32 phase's own arithmetic is
    FP32 and not counted."""
    sweeps, rots, checks = stats[:3]
    pairs = n * (n - 1) / 2
    qr1 = 2.0 * n * n * (s - n / 3.0)
    qr2 = 4.0 / 3.0 * n ** 3
    jac = (sweeps + checks) * pairs * 6.0 * n + rots * 12.0 * n
    prod = 0.0
    if len(stats) > 4 and stats[4] > 0:
        prod = 8.0 * n ** 3 + 2 * 6.0 * n ** 3 + (stats[6] if len(stats) > 6 else 0) * 2.0 * n ** 3
    return qr1 + qr2 + jac + prod + 4.0 * n * n * k


def launches_per_solve(stats):
    """Library kernels one solve of the headline launches (ns_solve_pipelined,
    nothing saved): the sketch (meta, chunk, reduce), the column order (3),
    both QRs (1, fused), X0 = R2^T and V = Q2 (2), the ring Jacobi, V = P Q2 V0 Vx
    and the extraction; when the FP32 phase runs (23 more): the phase, four
    products making V0 orthogonal and applying it, two completions of seven
    launches, the Gram-matrix check (2) and two copies."""
    return 12 + (23 if len(stats) > 4 and stats[4] > 0 else 0)


def cpu_baseline(A):
    """The oracle as it stands on the host cores: one full solve of the workload on
    one thread (best of 3), then as many concurrent solves as there are cores
    (threads; the C oracle releases the GIL), and the unsketched dense LAPACK
    SVD of A (numpy, best of 3) as the classical O(m n^2) context."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t1 = []
    out = None
    for _ in range(3):
        t0 = time.perf_counter()
        out = oracle.solve(oracle.SRHT, SEED, S, A, K_NULL)
        t1.append(time.perf_counter() - t0)
    best1 = min(t1)
    ta = []
    for _ in range(2):
        t0 = time.perf_counter()
        with concurrent.futures.ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(lambda _i: oracle.solve(oracle.SRHT, SEED, S, A, K_NULL)["status"], range(cores)))
        ta.append(time.perf_counter() - t0)
    tsvd = []
    for _ in range(3):
        t0 = time.perf_counter()
        np.linalg.svd(A, full_matrices=False)
        tsvd.append(time.perf_counter() - t0)
    return {"value": 1.0 / best1, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "one full oracle solve of the workload (m=2^20, n=256, s=1024, k=4) on one thread, "
                      "best of 3: %.2f s" % best1,
            "residual": oracle.residual(A, out["Vk"]),
            "all_cores": {"value": cores / min(ta), "unit": "solves/s", "cores": cores,
                          "sample": "%d concurrent oracle solves (one per core), best of 2: %.2f s" % (cores, min(ta))},
            "lapack_dense_svd": {"value": 1.0 / min(tsvd), "unit": "solves/s", "cores": cores,
                                 "sample": "numpy.linalg.svd of A (2^20 x 256, the unsketched O(m n^2) solve), "
                                           "best of 3: %.2f s" % min(tsvd)}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = make_workload(SEED)
    A = w["A"]
    import oracle
    oracle.build()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve(oracle.SRHT, SEED, S, A, K_NULL)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = len(times) / total
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(world),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": "full oracle solves of the workload, one per step"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class Timer:
    def __init__(self, torch, stream, dist, dev):
        self.torch, self.stream, self.dist, self.dev = torch, stream, dist, dev

    def __call__(self, fn, steps):
        torch, dist = self.torch, self.dist
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            fn()
        e1.record(self.stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms], device=self.dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms


def precision_input(torch, dev, seed):
    """The precision workload's A (m = 2^22, n = 512) on the GPU: sigma_1..510
    log-spaced from 1 to 1e-6, sigma_511 = sigma_512 = 1e-9, stored in FP32.
    A = U diag(sigma) V^T with U = G R^-1 the Cholesky-QR factor of a seeded
    Gaussian G (orthonormal to ~u for a Gaussian this tall), so A = G (R^-1
    diag(sigma) V^T) takes two FP64 GEMMs; V is the Q factor of a seeded
    Gaussian 512 x 512.  Input generation only (torch on the GPU)."""
    m, n, k = 1 << 22, 512, 2
    g = torch.Generator(device=dev).manual_seed(seed)
    G = torch.randn((n, m), generator=g, device=dev, dtype=torch.float64).t()  # column-major m x n
    R = torch.linalg.cholesky(G.t() @ G).t()                                  # upper, G^T G = R^T R
    V, _ = torch.linalg.qr(torch.randn((n, n), generator=g, device=dev, dtype=torch.float64))
    sig = torch.cat([torch.logspace(0, -6, n - k, dtype=torch.float64, device=dev),
                     torch.full((k,), 1e-9, dtype=torch.float64, device=dev)])
    Mr = torch.linalg.solve_triangular(R, torch.diag(sig) @ V.t(), upper=True)
    A64 = (G @ Mr).t().contiguous().t()
    del G
    A32 = A64.to(torch.float32).t().contiguous().t()
    del A64
    torch.cuda.empty_cache()
    return A32, V, sig, k


def precision_reference(torch, A32):
    """The FP64 reference for the FP32-stored A: R of a Householder QR of A (as
    FP64, cuSOLVER) and the SVD of R give sigma and the right singular vectors
    of A32 itself (the FP32 storage perturbs A by ~2^-24 ||A||, far above
    sigma_511 = 1e-9, so V's trailing columns are not A32's)."""
    R = torch.linalg.qr(A32.double(), mode="r")[1]
    _, sv, Vh = torch.linalg.svd(R)
    return sv, Vh.t()


def precision_accuracy(torch, A32, W, ref):
    """||A W||_F against the smallest possible (the trailing singular values of
    A32) and the sine to A32's trailing right singular subspace."""
    sv, Vr = ref
    k = W.shape[1]
    Wt = Vr[:, -k:]
    resid = float(torch.linalg.norm(A32.double() @ W))
    best = float(torch.sqrt((sv[-k:] ** 2).sum()))
    P = W - Wt @ (Wt.t() @ W)
    return {"residual_AW_F": resid, "residual_fp64_reference": best,
            "sine_to_fp64_reference": float(torch.linalg.matrix_norm(P, ord=2))}


def config_legs(torch, api, dev, timer, hbm_peak, bf16_peak, fp64_peak):
    """The other workloads, each with its own recipe (accuracy is checked
    against the oracle by the tests; here it is reported)."""
    from paper_2206_00975_gb300 import workloads
    out = {}
    stream = torch.cuda.current_stream()
    # ---- plain FP64: m = 4096, n = 32, s = 128, k = 1; single solves, and 1000 seeds batched
    w = workloads.plain(seed=0)
    A = api.colmajor(w["A"], device=dev)
    d = api.desc(api.NS_SRHT, s=128, seed=0)
    ws = api.workspace(d, 4096, 32, 1, dev)
    for _ in range(3):
        api.ns_solve(d, A, 1, save=False, ws=ws)
    ms = timer(lambda: api.ns_solve(d, A, 1, save=False, ws=ws), 50)
    Vk, _, _, _ = api.ns_solve(d, A, 1, save=False, ws=ws)
    probs = [{"A": A, "s": 128, "k": 1, "seed": i} for i in range(1000)]
    _, _, keep = api.ns_solve_batched(probs)
    msb = timer(lambda: api.ns_solve_batched(probs, ws=keep[2]), 3)
    out["plain_4096x32"] = {"solve_ms": ms / 50, "solves_per_s": 50 / (ms / 1e3),
                            "batched_1000_seeds_solves_per_s": 3000 / (msb / 1e3),
                            "residual_AV_F": float(api.ns_residual(A, Vk).item()),
                            "true_min_AV_F": float(w["sigma"][-1])}
    del probs, keep
    # ---- precision: m = 2^22, n = 512, A stored FP32 with the graded spectrum;
    # FP32-stream SRHT and 3 x BF16 Gaussian, s = 2048, FP64 QR / Jacobi
    A32, Vt, sig, k3 = precision_input(torch, dev, seed=3)
    ref3 = precision_reference(torch, A32)
    torch.cuda.empty_cache()
    m3, n3, s3 = A32.shape[0], A32.shape[1], 2048
    d32 = api.desc(api.NS_SRHT, s=s3, seed=0, prec=api.NS_PREC_FP32_STREAM)
    dg = api.desc(api.NS_GAUSSIAN, s=s3, seed=0, prec=api.NS_PREC_BF16X3)
    ws3 = api.workspace(d32, m3, n3, k3, dev)
    SA3 = api._empty_cm(s3, n3, dev)
    api.ns_sketch(d32, A32, SA=SA3, ws=ws3)
    ms32 = timer(lambda: api.ns_sketch(d32, A32, SA=SA3, ws=ws3), 5) / 5
    api.ns_solve(d32, A32, k3, save=False, ws=ws3)
    ms32s = timer(lambda: api.ns_solve(d32, A32, k3, save=False, ws=ws3), 3) / 3
    W32, sk32, _, st32 = api.ns_solve(d32, A32, k3, save=False, ws=ws3)
    acc32 = precision_accuracy(torch, A32, W32, ref3)
    del ws3
    torch.cuda.empty_cache()
    wsg = api.workspace(dg, m3, n3, k3, dev)
    api.ns_sketch(dg, A32, SA=SA3, ws=wsg)
    msg = timer(lambda: api.ns_sketch(dg, A32, SA=SA3, ws=wsg), 3) / 3
    Wg, skg, _, stg = api.ns_solve(dg, A32, k3, save=False, ws=wsg)
    msgs = timer(lambda: api.ns_solve(dg, A32, k3, save=False, ws=wsg), 2) / 2
    accg = precision_accuracy(torch, A32, Wg, ref3)
    b3 = m3 * n3 * 4 + s3 * n3 * 8
    mma_flops = 3 * 2.0 * s3 * m3 * n3
    out["precision_2^22x512"] = {
        "recipe": "sigma 1..1e-6 (510) + 2 x 1e-9, A = U diag(sigma) V^T stored FP32",
        "srht_fp32": {"sketch_ms": ms32, "sketch_gbs": b3 / (ms32 / 1e3) / 1e9,
                      "sketch_frac": b3 / (ms32 / 1e3) / 1e9 / hbm_peak, "solve_ms": ms32s,
                      "status": int(st32.item()), **acc32},
        "gaussian_bf16x3": {"sketch_ms": msg, "mma_tflops": mma_flops / (msg / 1e3) / 1e12,
                            "frac_of_bf16_peak": mma_flops / (msg / 1e3) / 1e12 / bf16_peak, "solve_ms": msgs,
                            "status": int(stg.item()), **accg}}
    del A32, SA3, wsg, W32, Wg
    torch.cuda.empty_cache()
    # ---- adjoint: m = 2^18, n = 128, k = 8, s = 512; L = ||W W^T Z||_F^2
    wa = workloads.adjoint(seed=0)
    A4 = api.colmajor(wa["A"], device=dev)
    d4 = api.desc(api.NS_SRHT, s=512, seed=0)
    ws4 = api.workspace(d4, 1 << 18, 128, 8, dev)
    Vk, sk, sv, _ = api.ns_solve(d4, A4, 8, ws=ws4)
    Z = torch.as_tensor(wa["W"], device=dev)
    dV = api.colmajor(2.0 * Z @ Z.T @ Vk)
    dA = api._empty_cm(1 << 18, 128, dev)
    api.ns_backward(d4, 1 << 18, 128, 8, sv, Vk, dV, dA=dA, ws=ws4)
    msf = timer(lambda: api.ns_solve(d4, A4, 8, save=sv, ws=ws4), 10) / 10
    msbw = timer(lambda: api.ns_backward(d4, 1 << 18, 128, 8, sv, Vk, dV, dA=dA, ws=ws4), 10) / 10
    out["adjoint_2^18x128"] = {"forward_ms": msf, "backward_ms": msbw,
                               "backward_write_gbs": (1 << 18) * 128 * 8 / (msbw / 1e3) / 1e9,
                               "backward_frac": (1 << 18) * 128 * 8 / (msbw / 1e3) / 1e9 / hbm_peak}
    del A4, ws4, dA
    torch.cuda.empty_cache()
    out["batched_tls_4096"] = batched_leg(torch, api, dev, timer)
    torch.cuda.empty_cache()
    # ---- AAA: 2^17 points, tanh(50 x), 100 iterations, 400-row sketch; eager vs CUDA graph
    x, f = workloads.aaa_points(seed=0, m=1 << 17, scale=50.0)
    xd, fd = torch.as_tensor(x, device=dev), torch.as_tensor(f, device=dev)
    r = api.ns_aaa_real(xd, fd, 100, 400, seed=0)
    torch.cuda.synchronize()
    wsa = r["_ws"]
    mse = timer(lambda: api.ns_aaa_real(xd, fd, 100, 400, seed=0, ws=wsa), 3) / 3
    s_cap = torch.cuda.Stream()
    s_cap.wait_stream(stream)
    with torch.cuda.stream(s_cap):
        api.ns_aaa_real(xd, fd, 100, 400, seed=0, ws=wsa, stream=s_cap)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s_cap, capture_error_mode="thread_local"):
        api.ns_aaa_real(xd, fd, 100, 400, seed=0, ws=wsa, stream=s_cap)
    graph.replay()
    torch.cuda.synchronize()
    msg2 = timer(lambda: graph.replay(), 3) / 3
    out["aaa_2^17_100it"] = {"eager_ms": mse, "graph_ms": msg2, "iterations_per_s_graph": 100 / (msg2 / 1e3),
                             "final_err": float(r["errmax"][-1].item())}
    return out


def batched_leg(torch, api, dev, timer):
    """Batched TLS: 4096 problems [X b], m_i ~ U{2^11..2^16}, n_i ~ U{8..128},
    X Gaussian, b = X x_true + 1e-3 noise (generated on the GPU), SRHT with
    s_i = 2(n_i + 1), k = 1: one batched call in FP64 and one with A in FP32
    (FP32-stream sketch), against a loop of single FP64 ns_solve calls."""
    from paper_2206_00975_gb300 import workloads
    ms_, ns_ = workloads.tls_batch_shapes(seed=0, batch=4096)
    g = torch.Generator(device=dev).manual_seed(5)
    probs, probs32, total = [], [], 0
    for i, (mi, ni) in enumerate(zip(ms_, ns_)):
        mi, ni = int(mi), int(ni)
        X = torch.randn((ni, mi), generator=g, device=dev, dtype=torch.float64).t()
        xt = torch.randn(ni, generator=g, device=dev, dtype=torch.float64)
        b = X @ xt + 1e-3 * torch.randn(mi, generator=g, device=dev, dtype=torch.float64)
        Xb = torch.empty((ni + 1, mi), device=dev, dtype=torch.float64).t()
        Xb[:, :ni] = X
        Xb[:, ni] = b
        probs.append({"A": Xb, "s": 2 * (ni + 1), "k": 1, "seed": i, "tls": True, "x_true": xt})
        total += mi * (ni + 1)
        del X
    _, st, keep = api.ns_solve_batched(probs[:64])
    outs, st, keep = api.ns_solve_batched(probs)
    ms64 = timer(lambda: api.ns_solve_batched(probs, ws=keep[2]), 2) / 2
    outs, st, keep = api.ns_solve_batched(probs, ws=keep[2])
    torch.cuda.synchronize()
    err = [float(torch.linalg.norm(o[2] - p["x_true"]) / torch.linalg.norm(p["x_true"])) for o, p in
           zip(outs[:256], probs[:256])]
    res = {"problems": len(probs), "input_gb_fp64": total * 8 / 1e9, "batched_fp64_ms": ms64,
           "batched_fp64_solves_per_s": len(probs) / (ms64 / 1e3),
           "status_nonzero_fp64": int((st != 0).sum().item()),
           "tls_relerr_median_first256": float(np.median(err))}
    # the per-problem FP64 loop on the first 256 problems, extrapolated
    sub = probs[:256]
    descs = [api.desc(api.NS_SRHT, s=p["s"], seed=p["seed"]) for p in sub]
    wss = [api.workspace(dd, p["A"].shape[0], p["A"].shape[1], 1, dev) for dd, p in zip(descs, sub)]

    def loop():
        for dd, p, wsp in zip(descs, sub, wss):
            api.ns_solve(dd, p["A"], 1, save=False, ws=wsp)
    loop()
    msl = timer(loop, 1) * len(probs) / len(sub)
    res["loop_fp64_solves_per_s_extrapolated"] = len(probs) / (msl / 1e3)
    del wss, keep
    torch.cuda.empty_cache()
    if getattr(api, "batched_supports_fp32", lambda: False)():
        for p in probs:
            p["A"] = p["A"].to(torch.float32).t().contiguous().t()
        outs32, st32, keep32 = api.ns_solve_batched(probs)
        ms32 = timer(lambda: api.ns_solve_batched(probs, ws=keep32[2]), 2) / 2
        outs32, st32, keep32 = api.ns_solve_batched(probs, ws=keep32[2])
        torch.cuda.synchronize()
        err32 = [float(torch.linalg.norm(o[2] - p["x_true"]) / torch.linalg.norm(p["x_true"])) for o, p in
                 zip(outs32[:256], probs[:256])]
        res.update({"input_gb_fp32": total * 4 / 1e9, "batched_fp32_stream_ms": ms32,
                    "batched_fp32_stream_solves_per_s": len(probs) / (ms32 / 1e3),
                    "status_nonzero_fp32": int((st32 != 0).sum().item()),
                    "tls_relerr_median_first256_fp32": float(np.median(err32))})
        del keep32
    del probs
    return res


def row_sharded_leg(torch, api, dev, dist, rank, world, args):
    """One A (the headline workload, the same seed on every rank) split by rows
    across the ranks: each rank forms its block's share of the SRHT sketch
    (ns_sketch_rows), one NCCL sum all-reduce of the s x n shares gives every
    rank the whole sketch, and every rank runs the dense stage.  One solve per
    step for the whole job (strong scaling of the sketch)."""
    from paper_2206_00975_gb300 import sharded
    w = make_workload(SEED)
    o, rows = sharded.row_partition(M, world)[rank]
    A_blk = torch.from_numpy(np.ascontiguousarray(w["A"][o:o + rows].T)).to(dev).t()
    del w
    d = api.desc(api.NS_SRHT, s=S, seed=SEED)
    ws_r = api.sketch_rows_workspace(d, M, o, max(rows, 1), N, dev)
    ws_d = api.workspace(d, M, N, K_NULL, dev)
    SA = api._empty_cm(S, N, dev)

    def step():
        sharded.sharded_sketch(d, A_blk, o, M, SA=SA, ws=ws_r)
        return api.ns_solve_sketched(d, SA, K_NULL, ws=ws_d)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    timer = Timer(torch, torch.cuda.current_stream(), dist, dev)
    ms = timer(step, args.steps)
    Vk, sk, _, st = step()
    torch.cuda.synchronize()
    return {"solves_per_s": args.steps / (ms / 1e3), "ms_per_solve": ms / args.steps, "rows_per_rank": rows,
            "scaling": "strong", "collective": "one NCCL all-reduce (sum) of the s x n FP64 shares per solve",
            "status": int(st.item()), "sigma_k": [float(x) for x in sk.cpu()]}


def hrht_moved_bytes(m, n, s):
    """DRAM bytes the two-pass H-RHT moves per sketch: A read once, the
    transformed blocks (int64, m' x n) written by pass 1 and read by pass 2,
    the hash table written once (pass 2 reads it from L2), the segment
    partials written and read, SA written."""
    mp = 1 << (m - 1).bit_length()
    blocks = max(mp // 4096, 1)
    want, nseg = max(16, -(-2048 // n)), 1
    while nseg < want and nseg < 64:
        nseg *= 2
    nseg = min(nseg, blocks)
    return 8 * m * n + 2 * 8 * max(mp, 4096) * n + 4 * mp + 2 * 8 * nseg * n * s + 8 * s * n


def profile_case(args, torch, api, dev):
    """One kernel family on a small case (a few GB at most), for ncu captures."""
    g = torch.Generator(device=dev).manual_seed(1)
    if args.case == "srht":        # 2^19 x 64 FP64 = 256 MiB (> L2)
        m, n, s = 1 << 19, 64, 1024
        A = torch.randn((n, m), generator=g, device=dev, dtype=torch.float64).t()
        d = api.desc(api.NS_SRHT, s=s, seed=0)
    elif args.case == "sparse":
        m, n, s = 1 << 19, 64, 1024
        A = torch.randn((n, m), generator=g, device=dev, dtype=torch.float64).t()
        d = api.desc(api.NS_SPARSE_SIGN, s=s, seed=0, zeta=8)
    elif args.case == "hrht":
        m, n, s = 1 << 19, 64, 1024
        A = torch.randn((n, m), generator=g, device=dev, dtype=torch.float64).t()
        d = api.desc(api.NS_HRHT, s=s, seed=0)
    elif args.case == "srht32":
        m, n, s = 1 << 20, 64, 2048
        A = torch.randn((n, m), generator=g, device=dev, dtype=torch.float32).t()
        d = api.desc(api.NS_SRHT, s=s, seed=0, prec=api.NS_PREC_FP32_STREAM)
    elif args.case == "gauss":
        m, n, s = 1 << 17, 512, 2048
        A = torch.randn((n, m), generator=g, device=dev, dtype=torch.float32).t()
        d = api.desc(api.NS_GAUSSIAN, s=s, seed=0, prec=api.NS_PREC_BF16X3)
    elif args.case == "fp64peak":  # FP64 throughput: cuBLAS DGEMM 8192^3 (2 n^3 flops), best of 5
        nn = 8192
        a = torch.randn((nn, nn), generator=g, device=dev, dtype=torch.float64)
        b = torch.randn((nn, nn), generator=g, device=dev, dtype=torch.float64)
        c = a @ b
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        print(json.dumps({"case": "fp64peak", "dgemm_n": nn, "ms": best, "tflops": 2.0 * nn ** 3 / (best / 1e3) / 1e12,
                          "sms": sms, "checksum": float(c[0, 0])}))
        return
    elif args.case == "dense":     # the at-scale dense stage on a Gaussian sketch
        n, s = N, S
        SA = torch.randn((n, s), generator=g, device=dev, dtype=torch.float64).t()
        d = api.desc(api.NS_SRHT, s=s, seed=0)
        ws = api.workspace(d, s, n, K_NULL, dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        for _ in range(args.steps):
            api.ns_solve_sketched(d, SA, K_NULL, status=status, ws=ws)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "n": n, "s": s, "steps": args.steps, "status": int(status.item())}))
        return
    else:
        raise SystemExit("unknown case " + args.case)
    ws = api.workspace(d, m, n, 1, dev)
    SAo = api._empty_cm(s, n, dev)
    for _ in range(args.steps):
        api.ns_sketch(d, A, SA=SAo, ws=ws)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "m": m, "n": n, "s": s, "steps": args.steps}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads (headline only)")
    ap.add_argument("--case", default=None,
                    help="profiling case: srht, sparse, hrht, srht32, gauss, dense, fp64peak")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2206_00975_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    from paper_2206_00975_gb300 import api
    dev = torch.device("cuda", local)
    if args.case:
        return profile_case(args, torch, api, dev)

    w = make_workload(SEED + rank)
    A_np = w["A"]
    A_host = torch.from_numpy(np.ascontiguousarray(A_np.T)).pin_memory().t()     # column-major, pinned
    A = A_host.to(dev, non_blocking=False)
    d = api.desc(api.NS_SRHT, s=S, seed=SEED)
    ws = api.workspace(d, M, N, K_NULL, dev)
    ws_dense = api.workspace(d, M, N, K_NULL, dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    save = torch.empty(api.save_size(S, N), dtype=torch.float64, device=dev)
    SA = api._empty_cm(S, N, dev)
    stream = torch.cuda.current_stream()
    timer = Timer(torch, stream, dist, dev)

    def solve(Ain):
        return api.ns_solve(d, Ain, K_NULL, save=save, status=status, ws=ws, stream=stream)

    for _ in range(args.warmup):
        Vk, sk, _, _ = solve(A)
        api.ns_sketch(d, A, SA=SA, ws=ws, stream=stream)
        api.ns_solve_sketched(d, SA, K_NULL, ws=ws_dense, stream=stream)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise SystemExit("solve status %d" % int(status.item()))

    # the headline: a stream of solves through ns_solve_pipelined, three in
    # flight, each lane's next sketch overlapping its dense stage past the QRs
    # (every step the same resident A; each problem is sketched and solved)
    ws_pipe = api.pipelined_workspace(d, M, N, dev)
    st_pipe = torch.zeros(args.steps, dtype=torch.int32, device=dev)

    def solve_stream():
        return api.ns_solve_pipelined(d, [A] * args.steps, K_NULL, status=st_pipe, ws=ws_pipe, stream=stream)

    for _ in range(args.warmup):
        Vks_p, sig_p, _ = solve_stream()
    torch.cuda.synchronize()
    if int(st_pipe.abs().max().item()) != 0 or not torch.equal(Vks_p[0], Vk):
        raise SystemExit("pipelined solve differs from ns_solve")

    # the same workload with the sparse-sign sketch (zeta = 8, s = 1024)
    dsp = api.desc(api.NS_SPARSE_SIGN, s=S, seed=SEED, zeta=8)
    ws_sp = api.workspace(dsp, M, N, K_NULL, dev)
    status_sp = torch.zeros(1, dtype=torch.int32, device=dev)

    def solve_sparse():
        return api.ns_solve(dsp, A, K_NULL, save=False, status=status_sp, ws=ws_sp, stream=stream)

    for _ in range(args.warmup):
        solve_sparse()
        api.ns_sketch(dsp, A, SA=SA, ws=ws_sp, stream=stream)
    torch.cuda.synchronize()

    # and with the H-RHT (the 1-hashing in place of the row sample, s = 1024)
    dh = api.desc(api.NS_HRHT, s=S, seed=SEED)
    ws_h = api.workspace(dh, M, N, K_NULL, dev)
    status_h = torch.zeros(1, dtype=torch.int32, device=dev)

    def solve_hrht():
        return api.ns_solve(dh, A, K_NULL, save=False, status=status_h, ws=ws_h, stream=stream)

    for _ in range(args.warmup):
        solve_hrht()
        api.ns_sketch(dh, A, SA=SA, ws=ws_h, stream=stream)
    torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        ms_pipe = timer(solve_stream, 1)
        ms_solve = timer(lambda: solve(A), args.steps)
        ms_sketch = timer(lambda: api.ns_sketch(d, A, SA=SA, ws=ws, stream=stream), args.steps)
        ms_dense = timer(lambda: api.ns_solve_sketched(d, SA, K_NULL, ws=ws_dense, stream=stream), args.steps)
        ms_solve_sp = timer(solve_sparse, args.steps)
        ms_sketch_sp = timer(lambda: api.ns_sketch(dsp, A, SA=SA, ws=ws_sp, stream=stream), args.steps)
        ms_solve_h = timer(solve_hrht, args.steps)
        ms_sketch_h = timer(lambda: api.ns_sketch(dh, A, SA=SA, ws=ws_h, stream=stream), args.steps)
    clocks = clk.summary()
    stats = api.jacobi_stats(d, M, N, ws_dense, sketched=True)

    # end to end through the public API: every step copies its A (2 GiB) from
    # pinned host memory and reads V_k and sigma_k back.  The host copy is the
    # contiguous (n, m) storage of the column-major A, split into E2E_PARTS
    # column ranges copied on as many streams (one copy engine each); two
    # device buffers let the copy of step i + 1 overlap the solve of step i.
    H = A_host.t()  # (n, m) contiguous, pinned
    Dbuf = [torch.empty_like(H, device=dev), torch.empty_like(H, device=dev)]
    Vk_host = torch.empty((K_NULL, N), dtype=torch.float64).pin_memory()
    sk_host = torch.empty(K_NULL, dtype=torch.float64).pin_memory()
    parts = [(N * q) // E2E_PARTS for q in range(E2E_PARTS + 1)]
    cstreams = [torch.cuda.Stream() for _ in range(E2E_PARTS)]
    ready = [[torch.cuda.Event() for _ in range(E2E_PARTS)] for _ in range(2)]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_steps = max(6, args.steps)

    def e2e_run(steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for cs in cstreams:
            cs.wait_stream(stream)
        for i in range(steps):
            b = i & 1
            for q, cs in enumerate(cstreams):
                with torch.cuda.stream(cs):
                    if i >= 2:
                        cs.wait_event(done[b])
                    Dbuf[b][parts[q]:parts[q + 1]].copy_(H[parts[q]:parts[q + 1]], non_blocking=True)
                    ready[b][q].record(cs)
            for q in range(E2E_PARTS):
                stream.wait_event(ready[b][q])
            Vk, sk, _, _ = solve(Dbuf[b].t())
            Vk_host.copy_(Vk.t(), non_blocking=True)
            sk_host.copy_(sk, non_blocking=True)
            done[b].record(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    e2e_run(2)  # warm-up
    ms_e2e = e2e_run(e2e_steps)
    e2e_ok = bool(np.isfinite(sk_host.numpy()).all() and np.isfinite(Vk_host.numpy()).all())

    # accuracy of the last solves
    Vk, sk, _, _ = solve(A)
    resid = float(api.ns_residual(A, Vk).item())
    Vk_sp, sk_sp, _, _ = solve_sparse()
    resid_sp = float(api.ns_residual(A, Vk_sp).item())
    torch.cuda.synchronize()
    if int(status_sp.item()) != 0:
        raise SystemExit("sparse-sign solve status %d" % int(status_sp.item()))
    Vk_h, _, _, _ = solve_hrht()
    resid_h = float(api.ns_residual(A, Vk_h).item())
    torch.cuda.synchronize()
    if int(status_h.item()) != 0:
        raise SystemExit("H-RHT solve status %d" % int(status_h.item()))

    n_ranks = world
    hbm_peak, bf16_peak, peak_kind = peaks()
    sketch_bytes = M * N * 8 + S * N * 8                # read A once, write SA
    t_sketch = ms_sketch / args.steps / 1e3
    t_dense = ms_dense / args.steps / 1e3
    sketch_gbs = sketch_bytes / t_sketch / 1e9
    sm_mhz = clocks.get("sm_mhz") or 1990.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = FP64_FLOPS_PER_CLK_SM * n_sm * sm_mhz * 1e6 / 1e12    # TFLOP/s at the sampled clock
    dflops = dense_flops(S, N, K_NULL, stats)
    dense_tf = dflops / t_dense / 1e12
    sketch_roof = {"bound": "hbm", "achieved": sketch_gbs, "peak": hbm_peak, "unit": "GB/s",
                   "frac": sketch_gbs / hbm_peak, "traffic": SRHT_TRAFFIC, "traffic_source": SRHT_TRAFFIC_SOURCE,
                   "kernel": "srht_f64_chunk256_kernel (ns_sketch)",
                   "peak_source": peak_kind, "algorithmic_bytes": sketch_bytes}
    dense_roof = {"bound": "alu", "achieved": dense_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                  "frac": dense_tf / fp64_peak, "traffic": None,
                  "kernel": "dense stage (column order, both Householder QRs in one fused launch with Q2 formed in "
                            "the second, FP32 Jacobi phase + FP64 products and two first-order completions, "
                            "Gram-matrix check, jacobi_ring from V = Q2 V0, extract) via ns_solve_sketched",
                  "peak_source": "derived: %d SMs x 4 FP64 flop/clk x sampled SM clock" % n_sm,
                  "algorithmic_flops": dflops, "jacobi_sweeps_rotations_checks": stats[:3],
                  "fp32_phase_sweeps_rotations": stats[4:6],
                  "completions_with_k4_and_gram_check": stats[6:8],
                  "jacobi_kernel": ("cluster ring, %d CTAs per cluster" % stats[3]) if stats[3] else "barrier-separated"}
    dominant = dense_roof if t_dense > t_sketch else sketch_roof
    line = {
        "metric": METRIC, "value": n_ranks * args.steps / (ms_pipe / 1e3), "unit": "solves/s", "n_gpus": n_ranks,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_pipe / args.steps, "higher_is_better": True,
        "mode": "ns_solve_pipelined: each step sketches and solves one problem; steps go round-robin to "
                "three lanes (three solves in flight), and within a lane the next sketch overlaps the dense "
                "stage past its QRs",
        "sequential": {"solves_per_s": n_ranks * args.steps / (ms_solve / 1e3), "ms_per_solve": ms_solve / args.steps,
                       "api": "ns_solve, one problem after the other on one stream"},
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(world),
        "roofline": dominant,
        "sketch_roofline": sketch_roof,
        "breakdown_ms": {"sketch": t_sketch * 1e3, "dense": t_dense * 1e3},
        "accuracy": {"residual_AV_F": resid, "sigma_k": [float(x) for x in sk.cpu()]},
        "sparse_sign": {"zeta": 8, "s": S, "solves_per_s": n_ranks * args.steps / (ms_solve_sp / 1e3),
                        "sketch_ms": ms_sketch_sp / args.steps,
                        "sketch_gbs": sketch_bytes / (ms_sketch_sp / args.steps / 1e3) / 1e9,
                        "sketch_frac": sketch_bytes / (ms_sketch_sp / args.steps / 1e3) / 1e9 / hbm_peak,
                        "residual_AV_F": resid_sp},
        "hrht": {"s": S, "solves_per_s": n_ranks * args.steps / (ms_solve_h / 1e3),
                 "sketch_ms": ms_sketch_h / args.steps,
                 "sketch_gbs": sketch_bytes / (ms_sketch_h / args.steps / 1e3) / 1e9,
                 "sketch_frac": sketch_bytes / (ms_sketch_h / args.steps / 1e3) / 1e9 / hbm_peak,
                 "moved_bytes_per_sketch": hrht_moved_bytes(M, N, S),
                 "moved_gbs": hrht_moved_bytes(M, N, S) / (ms_sketch_h / args.steps / 1e3) / 1e9,
                 "residual_AV_F": resid_h},
        "e2e": {"value": n_ranks * e2e_steps / (ms_e2e / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": M * N * 8, "d2h_bytes_per_step": (N * K_NULL + K_NULL) * 8,
                "overlap": "copy of step i+1 (E2E_PARTS streams) overlaps the solve of step i (two device buffers)",
                "results_finite": e2e_ok},
        "gpu_launches": launches_per_solve(stats) * args.steps,
        "clocks": clocks,
    }
    if world > 1:
        line["row_sharded"] = row_sharded_leg(torch, api, dev, dist, rank, world, args)
    if rank == 0 and n_ranks == 1 and not args.no_configs:
        line["configs"] = config_legs(torch, api, dev, Timer(torch, stream, None, dev), hbm_peak, bf16_peak,
                                      fp64_peak)
    if rank == 0 and n_ranks == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A_np)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
