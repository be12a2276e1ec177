"""H_W kernels (FP64, FP32) against the oracle, through the C ABI (GPU)."""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl, freefield, wilson
from tests.gpu_common import M0, make_ctx, rel, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,bc_t,nrhs", [((4, 4, 4, 4), -1, 1), ((3, 5, 4, 6), -1, 2), ((6, 4, 2, 5), 1, 3),
                                            ((8, 8, 8, 8), -1, 2), ((1, 2, 3, 4), -1, 2), ((5, 1, 1, 3), 1, 1)])
def test_hw_fp64_matches_oracle(gpu_lib, dims, bc_t, nrhs):
    import torch

    ctx, U = make_ctx(gpu_lib, dims, 0.5, 11, bc_t=bc_t)
    psi = S.gaussian_spinor(dims, 12, n=nrhs)
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    ctx.apply_HW(to_dev(psi), out, nrhs, gpu_lib.OV_FP64)
    got = to_host(out)
    for k in range(nrhs):
        want = cimpl.hw_apply(U, psi[k], M0, bc_t=bc_t)
        assert np.abs(got[k] - want).max() <= 1e-14 * np.abs(want).max()
    # independent check of the oracle route on one case: NumPy restatement
    if dims == (4, 4, 4, 4):
        assert np.abs(got[0] - wilson.apply_HW(U, psi[0], M0, bc_t=float(bc_t))).max() < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (5, 3, 4, 6), (16, 16, 16, 16), (1, 2, 3, 4)])
def test_hw_fp32_matches_oracle(gpu_lib, dims):
    import torch

    ctx, U = make_ctx(gpu_lib, dims, 0.5, 21)
    psi = S.gaussian_spinor(dims, 22)
    out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    ctx.apply_HW(to_dev(psi.astype(np.complex64)), out, 1, gpu_lib.OV_FP32)
    want = cimpl.hw_apply(U, psi.astype(np.complex64).astype(np.complex128), M0)
    assert rel(to_host(out).astype(np.complex128), want) < 2e-6


def test_hw_free_field_16x32(gpu_lib):
    """U = 1 at the production lattice size 16^3 x 32: momentum-space closed form."""
    import torch

    dims = (16, 16, 16, 32)
    ctx, _ = make_ctx(gpu_lib, dims, 0.0, 0)
    psi = S.gaussian_spinor(dims, 31)
    out = torch.empty(psi.shape, dtype=torch.complex128, device="cuda")
    ctx.apply_HW(to_dev(psi), out, 1, gpu_lib.OV_FP64)
    want = freefield.apply_H(psi, M0)
    assert np.abs(to_host(out) - want).max() < 1e-12


def test_hw_hermitian_16x32(gpu_lib):
    import torch

    dims = (16, 16, 16, 32)
    ctx, _ = make_ctx(gpu_lib, dims, 0.6, 41)
    a = S.gaussian_spinor(dims, 42)
    b = S.gaussian_spinor(dims, 43)
    ab = np.stack([a, b])
    out = torch.empty(ab.shape, dtype=torch.complex128, device="cuda")
    ctx.apply_HW(to_dev(ab), out, 2, gpu_lib.OV_FP64)
    Ha, Hb = to_host(out)
    lhs, rhs = np.vdot(a, Hb), np.vdot(Ha, b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_hw_rejects_bad_arguments(gpu_lib):
    import torch

    ctx, _ = make_ctx(gpu_lib, (2, 2, 2, 2), 0.3, 1)
    x = torch.zeros((16, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(gpu_lib.OvError) as e:
        ctx.apply_HW(x, x, 1, gpu_lib.OV_FP64)  # aliasing
    assert e.value.code == gpu_lib.OV_ERR_INVALID_ARG
    ctx2 = gpu_lib.Context((2, 2, 2, 2))
    y = torch.zeros_like(x)
    with pytest.raises(gpu_lib.OvError) as e:
        ctx2.apply_HW(x, y, 1, gpu_lib.OV_FP64)  # no gauge
    assert e.value.code == gpu_lib.OV_ERR_NO_GAUGE


@pytest.mark.parametrize("variant", list(range(6)))
def test_hw_fp32_variants(gpu_lib, variant):
    """Every FP32 stencil variant (RHS tile, link compression, block size) against the
    oracle, with a right-hand-side count that leaves a ragged last tile."""
    import torch

    assert len(gpu_lib.hw32_variants()) == 6
    dims = (6, 4, 5, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.6, 71)
    ctx.set_hw32_variant(variant)
    nrhs = 7
    psi = S.gaussian_spinor(dims, 72, n=nrhs).astype(np.complex64)
    out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    ctx.apply_HW(to_dev(psi), out, nrhs, gpu_lib.OV_FP32)
    got = to_host(out).astype(np.complex128)
    for k in range(nrhs):
        want = cimpl.hw_apply(U, psi[k].astype(np.complex128), M0)
        assert rel(got[k], want) < 3e-6


def test_hw_fp32_autotuned_12rhs_16x32(gpu_lib):
    import torch

    dims = (16, 16, 16, 32)
    ctx, U = make_ctx(gpu_lib, dims, 0.6, 81)
    nrhs = 12
    psi = S.gaussian_spinor(dims, 82, n=nrhs).astype(np.complex64)
    out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    ctx.apply_HW(to_dev(psi), out, nrhs, gpu_lib.OV_FP32)
    got = to_host(out).astype(np.complex128)
    for k in (0, 11):
        assert rel(got[k], cimpl.hw_apply(U, psi[k].astype(np.complex128), M0)) < 3e-6
