"""Row-sharded sketch across ranks: each rank holds a block of rows of A, forms
its share of the sketch with ns_sketch_rows, and one sum all-reduce of the
s x n shares gives every rank the sketch of the whole A (SA = sum_p S_p A_p:
the columns of S go with the rows of A).  The dense stage (QR and Jacobi of
the s x n sketch) then runs on every rank.

This module only partitions rows and calls the library and the collective;
the sketch arithmetic runs in the library's kernels.
"""


def row_partition(m_total, world, align=4096):
    """Rows of each rank: a list of (row_offset, rows) covering 0..m_total-1 in
    order, boundaries on multiples of `align` (the SRHT's 4096-row blocks) so
    that no block is split between two ranks; trailing ranks may get no rows."""
    if m_total < 1 or world < 1:
        raise ValueError("need m_total >= 1 and world >= 1")
    nblk = -(-m_total // align)
    parts, start = [], 0
    for p in range(world):
        blocks = nblk // world + (1 if p < nblk % world else 0)
        end = min(start + blocks * align, m_total)
        parts.append((start, end - start))
        start = end
    return parts


def sharded_sketch(d, A_local, row_offset, m_total, group=None, sketch_rows=None, all_reduce=None, SA=None,
                   ws=None, stream=None):
    """The whole sketch SA (s x n) on every rank from this rank's rows
    A_local = A[row_offset:row_offset + rows, :].

    sketch_rows(d, A_local, row_offset, m_total, SA) -> this rank's share (default:
    the library's ns_sketch_rows); all_reduce(tensor) sums over the group (default:
    torch.distributed.all_reduce with SUM).  A rank without rows contributes zeros."""
    import torch
    if sketch_rows is None:
        from . import api

        def sketch_rows(dd, A, o, m, out):
            return api.ns_sketch_rows(dd, A, o, m, SA=out, ws=ws, stream=stream)
    if all_reduce is None:
        import torch.distributed as dist

        def all_reduce(t):
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return t
    n = A_local.shape[1]
    if SA is None:
        SA = torch.empty((n, d.s), dtype=torch.float64, device=A_local.device).t()
    if A_local.shape[0] > 0:
        SA = sketch_rows(d, A_local, row_offset, m_total, SA)
    else:
        SA.zero_()
    return all_reduce(SA)
