#!/usr/bin/env python
"""Benchmark of the sketch-and-solve null-space hot path (Algorithm 1) on GB300.

Workload (one step = one full solve): A = U diag(sigma) V^T with m = 2^20,
n = 256, sigma_1..252 log-spaced from 1 to 1e-6 and a 4-dimensional exact null
space; SRHT sketch with s = 1024; FP64 QR and one-sided Jacobi SVD; the k = 4
trailing right singular vectors.  A (2 GiB) is larger than L2, so every step
streams it from HBM.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

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
METRIC = "null-space solves/s and sketch HBM GB/s (% of peak) at stated ||AV||_F accuracy"
WORKLOAD = "at_scale: m=2^20 n=256 FP64 column-major, sigma log-spaced 1..1e-6 + 4 exact zeros, SRHT s=1024, k=4"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    w = make_workload(SEED + rank)
    A_np = w["A"]
    dev = torch.device("cuda", local)
    A_host = torch.from_numpy(np.ascontiguousarray(A_np.T)).pin_memory().t()     # column-major, pinned
    A = A_host.to(dev, non_blocking=False)
    d = api.desc(api.NS_SRHT, s=S, seed=SEED)
    ws = api.workspace(d, M, N, K_NULL, dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    save = torch.empty(api.save_size(S, N), dtype=torch.float64, device=dev)
    SA = api._empty_cm(S, N, dev)
    stream = torch.cuda.current_stream()

    def solve(Ain):
        return api.ns_solve(d, Ain, K_NULL, save=save, status=status, ws=ws, stream=stream)

    for _ in range(args.warmup):
        Vk, sk, _, _ = solve(A)
        api.ns_sketch(d, A, SA=SA, ws=ws, stream=stream)
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise SystemExit("solve status %d" % int(status.item()))

    def timed(fn, steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
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

    with ClockSampler(local) as clk:
        ms_solve = timed(lambda: solve(A), args.steps)
        ms_sketch = timed(lambda: api.ns_sketch(d, A, SA=SA, ws=ws, stream=stream), args.steps)
        ms_solve_sp = timed(solve_sparse, args.steps)
        ms_sketch_sp = timed(lambda: api.ns_sketch(dsp, A, SA=SA, ws=ws_sp, stream=stream), args.steps)
    clocks = clk.summary()

    # end to end through the public API: pinned host A in, V_k and sigma_k back to host
    Vk_host = torch.empty((K_NULL, N), dtype=torch.float64).pin_memory()
    sk_host = torch.empty(K_NULL, dtype=torch.float64).pin_memory()
    A_stage = torch.empty_like(A)

    def e2e_step():
        A_stage.copy_(A_host, non_blocking=True)
        Vk, sk, _, _ = solve(A_stage)
        Vk_host.copy_(Vk.t(), non_blocking=True)
        sk_host.copy_(sk, non_blocking=True)

    e2e_steps = max(3, args.steps // 3)
    ms_e2e = timed(e2e_step, e2e_steps)

    # accuracy of the last solve
    Vk, sk, _, _ = solve(A)
    resid = float(api.ns_residual(A, Vk).item())
    Vk_sp, sk_sp, _, _ = solve_sparse()
    resid_sp = float(api.ns_residual(A, Vk_sp).item())
    torch.cuda.synchronize()
    if int(status_sp.item()) != 0:
        raise SystemExit("sparse-sign solve status %d" % int(status_sp.item()))

    n_ranks = world
    sketch_bytes = M * N * 8 + S * N * 8                # read A once, write SA
    t_solve = ms_solve / 1e3
    value = n_ranks * args.steps / t_solve
    hbm_peak, peak_kind = peaks()
    sketch_gbs = sketch_bytes / (ms_sketch / args.steps / 1e3) / 1e9
    dense_ms = (ms_solve - ms_sketch) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": n_ranks, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_solve / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "input larger than L2 (2 GiB A per step)", "parallelism":
                   "replicas" if n_ranks > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": sketch_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": sketch_gbs / hbm_peak, "traffic": None, "kernel": "SRHT sketch (ns_sketch)",
                     "peak_source": peak_kind},
        "breakdown_ms": {"sketch": ms_sketch / args.steps, "qr_jacobi_extract": dense_ms},
        "accuracy": {"residual_AV_F": resid, "sigma_k": [float(x) for x in sk.cpu()]},
        "sparse_sign": {"zeta": 8, "s": S, "solves_per_s": n_ranks * args.steps / (ms_solve_sp / 1e3),
                        "sketch_ms": ms_sketch_sp / args.steps,
                        "sketch_gbs": sketch_bytes / (ms_sketch_sp / args.steps / 1e3) / 1e9,
                        "sketch_frac": sketch_bytes / (ms_sketch_sp / args.steps / 1e3) / 1e9 / hbm_peak,
                        "residual_AV_F": resid_sp},
        "e2e": {"value": n_ranks * e2e_steps / (ms_e2e / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": M * N * 8, "d2h_bytes_per_step": (N * K_NULL + K_NULL) * 8},
        "gpu_launches": 6 * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and n_ranks == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A_np)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
