"""Sharding of the quadrature across processes (one GPU per process).

The resolvents of different nodes are independent (the paper splits the contour
points over MPI processes, Sec. "Numerical experiments").  With a node shard per rank,
each rank forms its partial sum c0_r b + sum_{j in shard} c_j (z_j - H)^-1 b and one
sum-allreduce gives S_N b; c0 is carried by rank 0 only.  Every rank repeats the
Krylov matrix-vector products of its own solve (the mat-vec is not split), so this
pays when the per-node work dominates, as in the paper's setting.

Independent sources need no exchange at all: ``source_shard`` splits them.
"""
from __future__ import annotations

import numpy as np


def contiguous_range(n: int, rank: int, world: int):
    """[lo, hi) of a contiguous, balanced split of n items over world ranks."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def node_shard(z, c, c0, rank: int, world: int):
    """This rank's nodes and coefficients, and its share of c0 (all of it on rank 0).

    Conjugate pairs (z_j, conj z_j) stay together when the list is ordered as the
    trapezoid rule of Eq. 7 orders it (pairs j, N+1-j): the split is over pair indices,
    so every rank's partial operator is hermitian by itself."""
    z = np.asarray(z, dtype=np.complex128)
    c = np.asarray(c, dtype=np.complex128)
    n = len(z)
    npair = (n + 1) // 2
    lo, hi = contiguous_range(npair, rank, world)
    idx = []
    for p in range(lo, hi):
        idx.append(p)
        q = n - 1 - p
        if q != p:
            idx.append(q)
    idx = np.array(sorted(idx), dtype=np.int64)
    return z[idx], c[idx], (complex(c0) if rank == 0 else 0j)


def source_shard(nsrc: int, rank: int, world: int):
    """[lo, hi) of the sources this rank processes (no exchange needed)."""
    return contiguous_range(nsrc, rank, world)


def allreduce_sum(t, group=None):
    """In-place sum over the ranks of a torch tensor (complex tensors as real pairs)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return t
    view = torch.view_as_real(t) if t.is_complex() else t
    dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
    return t


def sgn_sharded(ctx, b, opts=None, group=None):
    """S_N b with the nodes of ctx's contour split over the ranks of ``group``.

    ctx: a ``lib.Context`` on this rank's GPU with the gauge field and the full contour
    set (identical on every rank).  Returns S_N b on every rank.  Every arithmetic step
    runs in the library (ov_set_contour with this rank's share, ov_sgn_HW_apply); the
    only exchange is the sum-allreduce."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    z, c, c0 = ctx.get_contour()
    zr, cr, c0r = node_shard(z, c, c0, rank, world)
    out = torch.empty_like(b)
    nrhs = b.numel() // (12 * ctx.V)
    try:
        # a rank with no nodes sets an empty node list: the library then forms c0_r b
        ctx.set_contour(zr, cr, c0r)
        ctx.sgn(b, out, nrhs, opts)
    finally:
        ctx.set_contour(z, c, c0)
    return allreduce_sum(out, group)
