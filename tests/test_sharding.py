"""Node and source sharding over ranks (host logic), world size 2 with gloo on the CPU.

Each rank computes its partial sum of Eq. 7 with the oracle (the GPU library is not
available here), using the shard and allreduce of paper_2204_01583_gb300.parallel; the
allreduced result must equal the full quadrature."""
import os
import socket

import numpy as np
import pytest

from paper_2204_01583_gb300 import parallel


def test_contiguous_ranges_cover_exactly():
    for n in (0, 1, 5, 64, 65):
        for w in (1, 2, 3, 8):
            got = [parallel.contiguous_range(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[k][1] == got[k + 1][0] for k in range(w - 1))
            assert max(h - l for l, h in got) - min(h - l for l, h in got) <= 1


def test_node_shard_keeps_conjugate_pairs():
    from oracle import contour

    z, c, c0 = contour.single_contour(10, 3.0, 3.0, 0.3)
    seen = []
    for r in range(3):
        zr, cr, c0r = parallel.node_shard(z, c, c0, r, 3)
        # closed under conjugation (the nodes of a pair differ in the last bit)
        assert all(np.abs(zr - np.conj(zj)).min() < 1e-12 for zj in zr)
        assert (c0r == c0) == (r == 0)
        seen += list(zr)
    assert len(seen) == len(z) and all(np.abs(np.array(seen) - zj).min() == 0 for zj in z)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import synthetic as S
    from oracle import contour, sign, wilson

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims = (2, 2, 2, 4)
        U = S.su3_links(dims, 0.5, 901)
        b = S.gaussian_spinor(dims, 902)
        H = wilson.dense_HW(U, 1.6)
        z, c, c0 = contour.single_contour(16, 3.3, 3.3, 0.3)
        zr, cr, c0r = parallel.node_shard(z, c, c0, rank, world)
        part = sign.sign_apply_dense(H, b.reshape(-1), zr, cr, c0r)
        t = torch.from_numpy(part.copy())
        parallel.allreduce_sum(t)
        full = sign.sign_apply_dense(H, b.reshape(-1), z, c, c0)
        q.put((rank, float(np.linalg.norm(t.numpy() - full) / np.linalg.norm(full))))
    finally:
        dist.destroy_process_group()


def test_node_sharded_sum_world2_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert set(res) == {0, 1}
    assert max(res.values()) < 1e-13
