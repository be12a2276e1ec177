"""Shared helpers for the GPU tests: seeded workloads and tensor conversions."""
from __future__ import annotations

import numpy as np

import synthetic as S

M0 = 1.6


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def to_host(t):
    return t.detach().cpu().numpy()


def make_ctx(lib, dims, eps, seed, bc_t=-1, m0=M0):
    U = S.su3_links(dims, eps, seed) if eps > 0 else S.unit_links(dims)
    ctx = lib.Context(dims, bc_t=bc_t, m0=m0)
    ctx.set_gauge(to_dev(U))
    return ctx, U


def rel(a, b):
    """Relative difference of a from b, the larger of the 2-norm ratio ||a - b|| / ||b|| and
    the element-wise ratio max |a - b| / max |b|: an error confined to a few sites is not
    averaged away over the lattice, and a small error spread over every site is not hidden
    behind one large element."""
    d = np.abs(np.asarray(a) - np.asarray(b)).ravel()
    bb = np.abs(np.asarray(b)).ravel()
    return float(max(np.linalg.norm(d) / np.linalg.norm(bb), d.max() / bb.max()))


def rel_per_source(a, b):
    """rel() of every source (leading axis) separately."""
    return [rel(a[k], b[k]) for k in range(b.shape[0])]


def sgn_gpu(ctx, b, nrhs=None, **opts):
    import torch

    bd = to_dev(b)
    out = torch.empty_like(bd)
    n = nrhs if nrhs is not None else (b.shape[0] if b.ndim == 7 else 1)
    st = ctx.sgn(bd, out, n, ctx.opts(**opts) if opts else None)
    torch.cuda.synchronize()
    return to_host(out), st
