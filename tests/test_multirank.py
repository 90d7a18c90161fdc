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



class _Desc:
    def __init__(self, kind, s, seed, zeta=8):
        self.kind, self.s, self.seed, self.zeta = kind, s, seed, zeta


def _sharded_rank(rank, world, port, kind, out):
    """One gloo rank of the row-sharded sketch: its rows' share computed by the
    oracle (the sketch of A with every row outside the rank's block zeroed),
    then the host driver's sum all-reduce."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2206_00975_gb300 import sharded
    m, n, s, seed = 3 * 4096 + 777, 5, 96, 11
    A = np.random.default_rng(4).integers(-9, 10, size=(m, n)).astype(np.float64)
    o, rows = sharded.row_partition(m, world)[rank]

    def share(d, A_loc, off, m_total, SA):
        Az = np.zeros((m_total, A_loc.shape[1]))
        Az[off:off + A_loc.shape[0]] = A_loc.numpy()
        part = oracle.sketch(d.kind, d.seed, d.s, Az, zeta=d.zeta)
        SA.copy_(torch.from_numpy(part))
        return SA
    d = _Desc(kind, s, seed)
    SA = sharded.sharded_sketch(d, torch.from_numpy(np.asfortranarray(A[o:o + rows])), o, m, sketch_rows=share)
    full = oracle.sketch(kind, seed, s, A)
    out.put((rank, o, rows, float(np.max(np.abs(SA.numpy() - full))), float(np.max(np.abs(full)))))
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", [0, 1])   # SRHT, sparse sign
def test_row_sharded_sketch_over_gloo(kind):
    # two ranks, each with its block of rows (block-aligned boundary), one sum
    # all-reduce of the s x n shares: every rank ends with the whole sketch
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_rank, args=(r, 2, port, kind, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[:3] for g in got] == [(0, 0, 2 * 4096), (1, 2 * 4096, 4096 + 777)]
    for g in got:   # integer data: the shares add up to the sketch up to the scale's rounding
        assert g[3] <= 1e-13 * g[4]


def test_row_partition_covers_the_rows_on_block_boundaries():
    sys.path.insert(0, ROOT)
    from paper_2206_00975_gb300 import sharded
    for m, world in ((1 << 20, 4), (3 * 4096 + 5, 2), (1000, 3), (5 * 4096, 8)):
        parts = sharded.row_partition(m, world)
        assert len(parts) == world
        assert parts[0][0] == 0 and sum(r for _, r in parts) == m
        for (o, r), (o2, _) in zip(parts, parts[1:]):
            assert o + r == o2 and o2 % 4096 == 0 or o2 == m
