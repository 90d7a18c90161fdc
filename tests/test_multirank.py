"""The N > 1 host path of bench.py on CPU ranks over gloo (world size 2).

With --gpus N every rank solves its own replica of the workload: there is no
collective on the data path, only the timing protocol. Each timed region is
bracketed by barriers on every rank, and every rank then reports the slowest
rank's time (an all-reduce MAX), which gives the whole-job throughput. The
reference arm runs on rank 0 alone. No GPU is involved: Timer receives a
stand-in for torch.cuda whose events report a rank-dependent time, and a real
gloo process group.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Event:
    def __init__(self, ms):
        self.ms = ms

    def record(self, stream):
        pass

    def elapsed_time(self, end):
        return self.ms


class _Cuda:
    def __init__(self, ms, log):
        self.ms, self.log = ms, log

    def synchronize(self):
        self.log.append("sync")

    def Event(self, enable_timing=False):
        return _Event(self.ms)


class _Torch:
    """torch with its cuda namespace replaced (events report a fixed time)."""

    def __init__(self, ms, log):
        self.cuda = _Cuda(ms, log)
        self.tensor = torch.tensor


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    log, calls = [], []
    timer = bench.Timer(_Torch(5.0 + 2.0 * rank, log), None, dist, "cpu")
    ms = timer(lambda: calls.append(1), 3)
    out.put((rank, ms, len(calls), log.count("sync")))
    dist.destroy_process_group()


def test_timer_takes_the_slowest_rank_over_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # rank 0 timed 5 ms, rank 1 7 ms: both report the maximum; each ran its
    # own 3 steps between two synchronisations
    assert got == [(0, 7.0, 3, 2), (1, 7.0, 3, 2)]


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 3

    # a rank other than 0 returns at once: no workload, no oracle
    assert bench.run_reference(Args(), 1, 2) is None
