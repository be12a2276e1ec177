"""Overlap solve x = D_ov(m_q)^-1 b (ov_overlap_solve) against the oracle's dense solve on
the same quadrature nodes, and by its true residual at 8^4 (GPU)."""
import numpy as np
import pytest

import synthetic as S
from oracle import sign, wilson
from tests.gpu_common import M0, make_ctx, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def _solve(ctx, b, m_q, nrhs, tol=1e-12, mode="fp64_2pass", inner_tol=1e-13, **kw):
    import torch

    bd = to_dev(b)
    x = torch.empty_like(bd)
    st = ctx.overlap_solve(m_q, bd, x, nrhs, ctx.opts(mode=mode, tol=inner_tol), tol=tol, **kw)
    torch.cuda.synchronize()
    return to_host(x), st


@pytest.mark.parametrize("mode", ["fp64_2pass", "f32x2"])
def test_overlap_solve_4x4_vs_dense_oracle(gpu_lib, mode):
    """4^4, eps 0.3, N_q = 32 (Lanczos placement), m_q = 0.1, a Gaussian and a zero source."""
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, S.seed_for("config1"))
    ctx.place_contour(32, steps=120)
    b = S.gaussian_spinor(dims, S.seed_for("overlap-solve.b"))
    bb = np.stack([b, np.zeros_like(b)])
    x, st = _solve(ctx, bb, 0.1, 2, mode=mode)
    assert st["converged"] == 1 and st["max_residual"] <= 1e-10
    assert np.all(x[1] == 0)
    z, c, c0 = ctx.get_contour()
    want = sign.overlap_solve_dense(wilson.dense_HW(U, M0), b, z, c, c0, 0.1).reshape(b.shape)
    assert rel(x[0], want) < 1e-10


def test_overlap_solve_ragged_vs_dense_oracle(gpu_lib):
    dims = (3, 2, 2, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.5, 721)
    ctx.set_contour_ellipse(24, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 722, n=3)
    x, st = _solve(ctx, b, 0.2, 3)
    z, c, c0 = ctx.get_contour()
    H = wilson.dense_HW(U, M0)
    for k in range(3):
        want = sign.overlap_solve_dense(H, b[k], z, c, c0, 0.2).reshape(b[k].shape)
        assert rel(x[k], want) < 1e-10


def test_overlap_solve_8x4_true_residual(gpu_lib):
    """8^4 config-2 links (eps 0.5, N_q = 64), m_q = 0.1: the returned x satisfies
    ||b - D x|| / ||b|| <= 1e-10, checked with a separate overlap apply."""
    import torch

    dims = (8, 8, 8, 8)
    ctx, U = make_ctx(gpu_lib, dims, 0.5, S.seed_for("config2"))
    ctx.place_contour(64, steps=150)
    b = S.gaussian_spinor(dims, S.seed_for("config2.b"))
    x, st = _solve(ctx, b[None], 0.1, 1, mode="f32x2")
    assert st["converged"] == 1 and st["max_residual"] <= 1e-10
    Dx = torch.empty_like(to_dev(x))
    ctx.overlap(0.1, to_dev(x), Dx, 1, ctx.opts(mode="fp64_2pass", tol=1e-13))
    assert rel(to_host(Dx)[0], b) <= 1e-10


def test_overlap_solve_edge_cases(gpu_lib):
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 731)
    ctx.set_contour_ellipse(16, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 732)
    # m_q = 1: D = 1, one iteration gives x = b
    x, st = _solve(ctx, b[None], 1.0, 1)
    assert rel(x[0], b) < 1e-12 and st["iterations"] == 1
    # iteration cap -> NOT_CONVERGED with the last iterate
    bd = to_dev(b)
    xd = torch.empty_like(bd)
    st = ctx.overlap_solve(0.1, bd, xd, 1, ctx.opts(tol=1e-12), tol=1e-12, max_iter=2, allow_not_converged=True)
    assert st["status"] == gpu_lib.OV_ERR_NOT_CONVERGED and st["iterations"] == 2
    # bad arguments
    with pytest.raises(gpu_lib.OvError):
        ctx.overlap_solve(0.1, bd, xd, 1, tol=0.0)
    with pytest.raises(gpu_lib.OvError):
        ctx.overlap_solve(0.1, bd, bd, 1)
    # host buffers (inner host_io) give the same x
    hb = torch.from_numpy(b.copy())
    hx = torch.empty_like(hb)
    ctx.overlap_solve(0.2, hb, hx, 1, ctx.opts(tol=1e-13, host_io=True), tol=1e-12)
    xd2 = torch.empty_like(bd)
    ctx.overlap_solve(0.2, bd, xd2, 1, ctx.opts(tol=1e-13), tol=1e-12)
    assert np.array_equal(hx.numpy(), to_host(xd2))
    # page-locked host buffers (read and written by kernels, not the copy engine)
    pb, px = hb.pin_memory(), torch.empty_like(hb).pin_memory()
    ctx.overlap_solve(0.2, pb, px, 1, ctx.opts(tol=1e-13, host_io=True), tol=1e-12)
    assert np.array_equal(px.numpy(), to_host(xd2))
