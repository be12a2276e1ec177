"""Adjoint of sgn(H_W) b: source gradient and SU(3) link force (ov_sgn_vjp, ov_overlap_vjp)
against the oracle and central finite differences, and the autograd Function (GPU)."""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl, contour, force, sign, wilson
from tests.gpu_common import M0, make_ctx, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


def _vjp(gpu_lib, ctx, eta, b, **kw):
    import torch

    gb = torch.empty_like(to_dev(b))
    F = torch.empty((4,) + b.shape[:4] + (8,), dtype=torch.float64, device="cuda")
    st = ctx.sgn_vjp(to_dev(eta), to_dev(b), gb, F, ctx.opts(tol=1e-13, **kw))
    torch.cuda.synchronize()
    return to_host(gb), to_host(F), st


def test_force_matches_oracle_formula_small(gpu_lib):
    """2x2x2x4 lattice: the whole force array against the oracle's dense-resolvent force."""
    dims = (2, 2, 2, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.4, 601)
    ctx.set_contour_ellipse(16, 3.3, 3.3, 0.3)
    b = S.gaussian_spinor(dims, 602)
    eta = S.gaussian_spinor(dims, 603)
    gb, F, st = _vjp(gpu_lib, ctx, eta, b)
    z, c, c0 = ctx.get_contour()
    H = wilson.dense_HW(U, M0)
    y = sign.resolvents_dense(H, b.reshape(-1), z).reshape((len(z),) + b.shape)
    xi = sign.resolvents_dense(H, eta.reshape(-1), z.conj()).reshape((len(z),) + b.shape)
    Fo = force.link_force(U, y, xi, c)
    assert np.abs(F - Fo).max() <= 1e-10 * np.abs(Fo).max()
    go = force.source_gradient(xi, eta, c, c0)
    assert rel(gb, go) < 1e-10


@pytest.fixture(scope="module")
def config4(gpu_lib):
    """8^4, eps = 0.4, N_q = 48 (Lanczos placement); eta, b complex Gaussian."""
    dims = (8, 8, 8, 8)
    ctx, U = make_ctx(gpu_lib, dims, 0.4, S.seed_for("config4"))
    ctx.place_contour(48, steps=150)
    b = S.gaussian_spinor(dims, S.seed_for("config4.b"))
    eta = S.gaussian_spinor(dims, S.seed_for("config4.eta"))
    gb, F, st = _vjp(gpu_lib, ctx, eta, b)
    return ctx, U, b, eta, gb, F, st


def test_config4_source_gradient_vs_oracle(gpu_lib, config4):
    ctx, U, b, eta, gb, F, st = config4
    z, c, c0 = ctx.get_contour()
    want, _, _ = cimpl.sign_apply(U, eta, z.conj(), c.conj(), np.conj(c0), M0, tol=1e-13)
    assert rel(gb, want) < 1e-10


def _loss(gpu_lib, ctx, U, b, eta, K):
    """L_K = Re<eta, S_N b> from exactly K Krylov steps: a smooth function of the links."""
    import torch

    ctx.set_gauge(to_dev(U))
    out = torch.empty_like(to_dev(b))
    ctx.sgn(to_dev(b), out, 1, ctx.opts(tol=1e-300, max_iter=K), allow_not_converged=True)
    return float(np.vdot(eta, to_host(out)).real)


@pytest.mark.parametrize("mu,site,a", [(0, (0, 1, 2, 3), 0), (3, (7, 0, 5, 1), 7), (1, (3, 3, 3, 3), 4),
                                       (2, (5, 6, 0, 2), 2)])
def test_config4_force_vs_finite_differences(gpu_lib, config4, mu, site, a):
    """Central differences of L = Re<eta, S_N b> under U -> exp(+-i h T_a) U at one link
    (h = 1e-4; the t = 7 case crosses the antiperiodic boundary), to 1e-6 relative.  Both
    sides run the same fixed number of Krylov steps, well past convergence, so the
    difference quotient is not polluted by a change of the stopping iteration."""
    ctx, U, b, eta, gb, F, st = config4
    K = st["iterations"] + 40
    h = 1e-4
    th = np.zeros(8)
    th[a] = h
    Up, Um = U.copy(), U.copy()
    Up[(mu,) + site] = force.exp_generator(th) @ U[(mu,) + site]
    Um[(mu,) + site] = force.exp_generator(-th) @ U[(mu,) + site]
    fd = (_loss(gpu_lib, ctx, Up, b, eta, K) - _loss(gpu_lib, ctx, Um, b, eta, K)) / (2 * h)
    ctx.set_gauge(to_dev(U))
    got = F[(mu,) + site + (a,)]
    assert abs(got - fd) <= 1e-6 * max(abs(fd), np.abs(F).max() * 1e-3)


def test_node_chunks_recompute_same_gradient(gpu_lib, config4):
    ctx, U, b, eta, gb, F, st = config4
    gb2, F2, st = _vjp(gpu_lib, ctx, eta, b, node_chunk=7)
    assert rel(gb2, gb) < 1e-12
    assert np.abs(F2 - F).max() <= 1e-12 * np.abs(F).max()


def test_overlap_vjp(gpu_lib):
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 611)
    ctx.set_contour_ellipse(24, 3.3, 3.3, 0.3)
    b = S.gaussian_spinor(dims, 612)
    eta = S.gaussian_spinor(dims, 613)
    m = 0.1
    gb = torch.empty_like(to_dev(b))
    F = torch.empty((4,) + b.shape[:4] + (8,), dtype=torch.float64, device="cuda")
    ctx.overlap_vjp(m, to_dev(eta), to_dev(b), gb, F, ctx.opts(tol=1e-13))
    eta5 = sign.g5(eta)
    gs, Fs, _ = _vjp(gpu_lib, ctx, eta5, b)
    assert rel(to_host(gb), 0.5 * (1 + m) * eta + 0.5 * (1 - m) * gs) < 1e-12
    assert np.abs(to_host(F) - 0.5 * (1 - m) * Fs).max() <= 1e-12 * np.abs(Fs).max()


def test_autograd_function(gpu_lib):
    """torch autograd through SignFunction: the b-gradient and link force of L = Re<eta, S b>
    equal the VJP entry point, and the b-gradient matches a finite difference."""
    import torch

    from paper_2204_01583_gb300 import ops

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 621)
    ctx.set_contour_ellipse(24, 3.3, 3.3, 0.3)
    b = to_dev(S.gaussian_spinor(dims, 622)).requires_grad_(True)
    eta = to_dev(S.gaussian_spinor(dims, 623))
    omega = torch.zeros(ops.force_shape(dims), dtype=torch.float64, device="cuda", requires_grad=True)
    opts = ctx.opts(tol=1e-13)
    out = ops.SignFunction.apply(b, omega, ctx, opts)
    L = torch.real(torch.vdot(eta.reshape(-1), out.reshape(-1)))
    L.backward()
    gb, F, _ = _vjp(gpu_lib, ctx, to_host(eta), to_host(b.detach()))
    assert rel(to_host(b.grad), gb) < 1e-13
    assert np.abs(to_host(omega.grad) - F).max() <= 1e-13 * np.abs(F).max()
    # dL = Re<grad, db>
    d = to_dev(S.gaussian_spinor(dims, 624))
    h = 1e-6
    with torch.no_grad():
        Lp = torch.real(torch.vdot(eta.reshape(-1), ops.sgn_apply(ctx, b + h * d, opts).reshape(-1)))
        Lm = torch.real(torch.vdot(eta.reshape(-1), ops.sgn_apply(ctx, b - h * d, opts).reshape(-1)))
    fd = float((Lp - Lm) / (2 * h))
    assert abs(fd - float(torch.real(torch.vdot(b.grad.reshape(-1), d.reshape(-1))))) < 1e-7 * abs(fd)


@pytest.mark.parametrize("mode,chunk", [("fp64_2pass", 0), ("fp64_2pass", 7), ("f32x2", 0), ("f32x2", 13)])
def test_coefficient_space_vjp_matches_vector_space(gpu_lib, config4, mode, chunk):
    """The gradient through a stored Lanczos basis (per-node solutions formed from it, chunk
    by chunk; FP64 or double-float vectors) equals the FP64 vector-space one to 1e-10."""
    ctx, U, b, eta, gb, F, st = config4
    gb2, F2, st2 = _vjp(gpu_lib, ctx, eta, b, mode=mode, node_chunk=chunk)
    assert rel(gb2, gb) < 1e-10
    assert np.abs(F2 - F).max() <= 1e-10 * np.abs(F).max()


def test_host_buffers_give_the_device_result(gpu_lib):
    """ov_sgn_vjp with host_io: pageable numpy buffers (copy engine) and page-locked torch
    buffers (read and written by kernels) give the device-buffer gradients bit for bit."""
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 621)
    ctx.set_contour_ellipse(24, 3.3, 3.3, 0.3)
    b = S.gaussian_spinor(dims, 622)
    eta = S.gaussian_spinor(dims, 623)
    gb, F, _ = _vjp(gpu_lib, ctx, eta, b)
    for pinned in (False, True):
        hb, he = torch.from_numpy(b.copy()), torch.from_numpy(eta.copy())
        hg = torch.empty_like(hb)
        hF = torch.empty((4,) + b.shape[:4] + (8,), dtype=torch.float64)
        if pinned:
            hb, he, hg, hF = hb.pin_memory(), he.pin_memory(), hg.pin_memory(), hF.pin_memory()
        ctx.sgn_vjp(he, hb, hg, hF, ctx.opts(tol=1e-13, host_io=True))
        assert np.array_equal(hg.numpy(), gb), pinned
        assert np.array_equal(hF.numpy(), F), pinned
