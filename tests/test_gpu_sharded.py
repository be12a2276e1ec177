"""Node-sharded S_N b through the library: two processes on the one GPU (GPU).

The paper spreads the contour points over processes ("Numerical experiments", Table 1).
parallel.sgn_sharded gives each rank its share of the nodes (conjugate pairs kept
together, c0 on rank 0), runs ov_sgn_HW_apply on that share and sums the partial results
over the ranks.  Here two ranks run as two processes on the same GPU with the gloo
backend; their kernels never wait on one another (the only exchange is the host-side
sum after both solves).  The summed result is checked against the per-node CGNR
oracle on the full contour, element by element and in norm.  With a two-node contour
rank 1 holds no node at all and contributes nothing but its (zero) share of c0, through
the library's empty-contour path.
"""
import os
import socket

import numpy as np
import pytest

import synthetic as S
from oracle import cimpl, contour
from tests.gpu_common import M0, rel

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cases():
    z16, c16, c016 = contour.single_contour(16, 3.4, 3.4, 0.3)
    z2 = np.array([1.0 + 1.5j, 1.0 - 1.5j])
    c2 = np.array([0.6 + 0.3j, 0.6 - 0.3j])
    return [(z16, c16, c016), (z2, c2, -0.5 + 0.0j)]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2204_01583_gb300 import lib, parallel

        U = S.su3_links(DIMS, 0.4, 1301)
        b = S.gaussian_spinor(DIMS, 1302, n=2)
        ctx = lib.Context(DIMS, bc_t=-1, m0=M0)
        ctx.set_gauge(torch.from_numpy(U).cuda())
        outs = []
        for z, c, c0 in _cases():
            ctx.set_contour(z, c, c0)
            for mode in ("fp64_2pass", "f32x2"):
                got = parallel.sgn_sharded(ctx, torch.from_numpy(b).cuda(), ctx.opts(mode=mode, tol=1e-12))
                torch.cuda.synchronize()
                outs.append(got.cpu().numpy())
            # the context's full contour is restored after the sharded call
            zz, cc, _ = ctx.get_contour()
            assert len(zz) == len(z)
        ctx.close()
        q.put((rank, outs))
    finally:
        dist.destroy_process_group()


def test_node_sharded_sum_through_library_world2():
    import torch.multiprocessing as mp

    U = S.su3_links(DIMS, 0.4, 1301)
    b = S.gaussian_spinor(DIMS, 1302, n=2)
    want = []
    for z, c, c0 in _cases():
        w, _, _ = cimpl.sign_apply_many(U, b, z, c, c0, M0, tol=1e-13)
        want += [w, w]  # the two modes
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in (0, 1):
        for got, w in zip(res[r], want):
            for k in range(2):
                assert rel(got[k], w[k]) < 1e-10, (r, k, rel(got[k], w[k]))
