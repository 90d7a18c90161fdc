#!/usr/bin/env python
"""Benchmark of the sketch-and-solve null-space hot path (Algorithm 1) on GB300.

Workload (one step = one full solve): A = U diag(sigma) V^T with m = 2^20,
n = 256, sigma_1..252 log-spaced from 1 to 1e-6 and a 4-dimensional exact null
space; SRHT sketch with s = 1024; FP64 pivoted QR, QR of R^T and one-sided
Jacobi SVD; the k = 4 trailing right singular vectors.  A (2 GiB) is larger
than L2, so every step streams it from HBM.  The same workload is also solved
with the sparse-sign sketch (zeta = 8).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
    python bench.py --extra          # also time the other workloads
    python bench.py --case NAME      # one kernel family on a small case (profiling)

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own replica of the workload (weak scaling; the path needs no collective).
"""
import argparse
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
# DRAM bytes of one srht_f64_chunk128_kernel launch at full size: the ncu capture of
# profiles/srht_f64_chunk_m2e19_n64.md (268.58 MB read + 3.03 MB written at
# m = 2^19, n = 64) scaled by the 8x the full launch processes; the kernel is
# unchanged since that capture.
SRHT_TRAFFIC = (268.58e6 + 3.03e6) * 8
SRHT_TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum at m=2^19 n=64, scaled x8"
METRIC = "null-space solves/s and sketch HBM GB/s (% of peak) at stated ||AV||_F accuracy"
WORKLOAD = "at_scale: m=2^20 n=256 FP64 column-major, sigma log-spaced 1..1e-6 + 4 exact zeros, SRHT s=1024, k=4"
FP64_FLOPS_PER_CLK_SM = 4.0   # 2 FP64 FMA per clock per SM (measured 597 GFMA/s at 1.99 GHz on 152 SMs)
N_SM = 152


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
    pivoted Householder QR of s x n, Householder QR of n x n, one-sided Jacobi
    (dot products 6n per visited pair, rotation of two columns of X and of V 12n),
    and the k trailing columns of V = P Q2 Vx (4 n^2 k)."""
    sweeps, rots, checks = stats[:3]
    pairs = n * (n - 1) / 2
    qr1 = 2.0 * n * n * (s - n / 3.0)
    qr2 = 4.0 / 3.0 * n ** 3
    jac = (sweeps + checks) * pairs * 6.0 * n + rots * 12.0 * n
    return qr1 + qr2 + jac + 4.0 * n * n * k


def cpu_baseline(A):
    """The oracle as it stands, one full solve of the same workload, single-threaded."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    out = oracle.solve(oracle.SRHT, SEED, S, A, K_NULL)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "one full oracle solve of the workload (m=2^20, n=256, s=1024, k=4), %.1f s" % dt,
            "residual": oracle.residual(A, out["Vk"])}


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
            "config": {"workload": WORKLOAD, "l2": "input larger than L2 (2 GiB)"},
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


def extra_workloads(torch, api, dev, timer, hbm_peak, bf16_peak):
    """Timings of the other workloads (opt-in; accuracy is covered by the tests)."""
    from paper_2206_00975_gb300 import workloads
    out = {}
    # plain FP64: m = 4096, n = 32, s = 128, k = 1; single solves and 1000 seeds batched
    w = workloads.plain(seed=0)
    A = api.colmajor(w["A"], device=dev)
    d = api.desc(api.NS_SRHT, s=128, seed=0)
    ws = api.workspace(d, 4096, 32, 1, dev)
    for _ in range(3):
        api.ns_solve(d, A, 1, save=False, ws=ws)
    ms = timer(lambda: api.ns_solve(d, A, 1, save=False, ws=ws), 50)
    probs = [{"A": A, "s": 128, "k": 1, "seed": i} for i in range(1000)]
    api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    out["plain_4096x32"] = {"solve_ms": ms / 50, "solves_per_s": 50 / (ms / 1e3),
                            "batched_1000_seeds_solves_per_s": 1000 / tb}
    # precision: m = 2^22, n = 512, A stored FP32; FP32-stream SRHT and Gaussian 3xBF16 (s = 2048)
    m3, n3, s3 = 1 << 22, 512, 2048
    g = torch.Generator(device=dev).manual_seed(3)
    A3 = torch.randn((n3, m3), generator=g, device=dev, dtype=torch.float32).t()
    d32 = api.desc(api.NS_SRHT, s=s3, seed=0, prec=api.NS_PREC_FP32_STREAM)
    dg = api.desc(api.NS_GAUSSIAN, s=s3, seed=0, prec=api.NS_PREC_BF16X3)
    ws3 = api.workspace(d32, m3, n3, 2, dev)
    wsg = api.workspace(dg, m3, n3, 2, dev)
    SA3 = api._empty_cm(s3, n3, dev)
    api.ns_sketch(d32, A3, SA=SA3, ws=ws3)
    api.ns_sketch(dg, A3, SA=SA3, ws=wsg)
    ms32 = timer(lambda: api.ns_sketch(d32, A3, SA=SA3, ws=ws3), 5)
    msg = timer(lambda: api.ns_sketch(dg, A3, SA=SA3, ws=wsg), 3)
    b3 = m3 * n3 * 4 + s3 * n3 * 8
    mma_flops = 3 * 2.0 * s3 * m3 * n3
    out["precision_2^22x512"] = {
        "srht_fp32_ms": ms32 / 5, "srht_fp32_gbs": b3 / (ms32 / 5 / 1e3) / 1e9,
        "srht_fp32_frac": b3 / (ms32 / 5 / 1e3) / 1e9 / hbm_peak,
        "gaussian_bf16x3_ms": msg / 3, "gaussian_mma_tflops": mma_flops / (msg / 3 / 1e3) / 1e12,
        "gaussian_frac_of_bf16_peak": mma_flops / (msg / 3 / 1e3) / 1e12 / bf16_peak}
    del A3, SA3, ws3, wsg
    torch.cuda.empty_cache()
    # adjoint: m = 2^18, n = 128, k = 8, s = 512
    wa = workloads.adjoint(seed=0)
    A4 = api.colmajor(wa["A"], device=dev)
    d4 = api.desc(api.NS_SRHT, s=512, seed=0)
    ws4 = api.workspace(d4, 1 << 18, 128, 8, dev)
    Vk, sk, sv, _ = api.ns_solve(d4, A4, 8, ws=ws4)
    Z = torch.as_tensor(wa["W"], device=dev)
    dV = api.colmajor(2.0 * Z @ Z.T @ Vk)
    dA = api._empty_cm(1 << 18, 128, dev)
    api.ns_backward(d4, 1 << 18, 128, 8, sv, Vk, dV, dA=dA, ws=ws4)
    msf = timer(lambda: api.ns_solve(d4, A4, 8, save=sv, ws=ws4), 10)
    msb = timer(lambda: api.ns_backward(d4, 1 << 18, 128, 8, sv, Vk, dV, dA=dA, ws=ws4), 10)
    out["adjoint_2^18x128"] = {"forward_ms": msf / 10, "backward_ms": msb / 10,
                               "backward_write_gbs": (1 << 18) * 128 * 8 / (msb / 10 / 1e3) / 1e9}
    # batched TLS: 4096 problems, m ~ U{2^11..2^16}, n ~ U{8..128}, [X b] FP64 generated on the GPU
    ms_, ns_ = workloads.tls_batch_shapes(seed=0, batch=4096)
    probs, total_bytes = [], 0
    for i, (mi, ni) in enumerate(zip(ms_, ns_)):
        Xb = torch.randn((int(ni) + 1, int(mi)), generator=g, device=dev, dtype=torch.float64).t()
        probs.append({"A": Xb, "s": 2 * (int(ni) + 1), "k": 1, "seed": i, "tls": True})
        total_bytes += int(mi) * (int(ni) + 1) * 8
    api.ns_solve_batched(probs[:64])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st, keep = api.ns_solve_batched(probs)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    # the per-problem loop on a 256-problem subset (same problems), extrapolated
    sub = probs[:256]
    t0 = time.perf_counter()
    for p in sub:
        dd = api.desc(api.NS_SRHT, s=p["s"], seed=p["seed"])
        api.ns_solve(dd, p["A"], 1, save=False)
    torch.cuda.synchronize()
    tl = (time.perf_counter() - t0) * len(probs) / len(sub)
    out["batched_tls_4096"] = {"batched_s": tb, "batched_solves_per_s": len(probs) / tb,
                               "loop_solves_per_s_extrapolated": len(probs) / tl, "input_gb": total_bytes / 1e9,
                               "status_nonzero": int((st != 0).sum().item())}
    del probs, keep
    torch.cuda.empty_cache()
    # AAA: 2^17 points, tanh(50 x), 100 iterations, 400-row sketch; eager vs CUDA graph
    x, f = workloads.aaa_points(seed=0, m=1 << 17, scale=50.0)
    xd, fd = torch.as_tensor(x, device=dev), torch.as_tensor(f, device=dev)
    r = api.ns_aaa_real(xd, fd, 100, 400, seed=0)
    torch.cuda.synchronize()
    wsa = r["_ws"]
    mse = timer(lambda: api.ns_aaa_real(xd, fd, 100, 400, seed=0, ws=wsa), 3)
    s_cap = torch.cuda.Stream()
    s_cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s_cap):
        api.ns_aaa_real(xd, fd, 100, 400, seed=0, ws=wsa, stream=s_cap)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s_cap, capture_error_mode="thread_local"):
        api.ns_aaa_real(xd, fd, 100, 400, seed=0, ws=wsa, stream=s_cap)
    graph.replay()
    torch.cuda.synchronize()
    msg2 = timer(lambda: graph.replay(), 3)
    out["aaa_2^17_100it"] = {"eager_ms": mse / 3, "graph_ms": msg2 / 3, "iterations_per_s_graph": 100 / (msg2 / 3e3),
                             "final_err": float(r["errmax"][-1].item())}
    return out


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
    ap.add_argument("--extra", action="store_true", help="also time the other workloads")
    ap.add_argument("--case", default=None, help="profiling case: srht, sparse, hrht, srht32, gauss, dense")
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
    fp64_peak = FP64_FLOPS_PER_CLK_SM * N_SM * sm_mhz * 1e6 / 1e12    # TFLOP/s at the sampled clock
    dflops = dense_flops(S, N, K_NULL, stats)
    dense_tf = dflops / t_dense / 1e12
    sketch_roof = {"bound": "hbm", "achieved": sketch_gbs, "peak": hbm_peak, "unit": "GB/s",
                   "frac": sketch_gbs / hbm_peak, "traffic": SRHT_TRAFFIC, "traffic_source": SRHT_TRAFFIC_SOURCE,
                   "kernel": "srht_f64_chunk128_kernel (ns_sketch)",
                   "peak_source": peak_kind, "algorithmic_bytes": sketch_bytes}
    dense_roof = {"bound": "alu", "achieved": dense_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                  "frac": dense_tf / fp64_peak, "traffic": None,
                  "kernel": "FP64 dense stage (column order, hqr_pipe x2 with Q2 formed in the second, jacobi_ring from V = Q2, extract) via ns_solve_sketched",
                  "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x sampled SM clock",
                  "algorithmic_flops": dflops, "jacobi_sweeps_rotations_checks": stats[:3],
                  "jacobi_kernel": ("cluster ring, %d CTAs per cluster" % stats[3]) if stats[3] else "barrier-separated"}
    dominant = dense_roof if t_dense > t_sketch else sketch_roof
    line = {
        "metric": METRIC, "value": n_ranks * args.steps / (ms_solve / 1e3), "unit": "solves/s", "n_gpus": n_ranks,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_solve / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "input larger than L2 (2 GiB A per step)", "parallelism":
                   "replicas" if n_ranks > 1 else "single GPU"},
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
        "gpu_launches": 17 * args.steps,
        "clocks": clocks,
    }
    if args.extra and rank == 0:
        line["extra"] = extra_workloads(torch, api, dev, Timer(torch, stream, None, dev), hbm_peak, bf16_peak)
    if rank == 0 and n_ranks == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A_np)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
