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


@pytest.mark.parametrize("variant", list(range(23)))
def test_hw_fp32_variants(gpu_lib, variant):
    """Every FP32 stencil variant (RHS tile, link compression, block size) against the
    oracle, with a right-hand-side count that leaves a ragged last tile."""
    import torch

    assert len(gpu_lib.hw32_variants()) == 23
    code = gpu_lib.hw32_variants()[variant][1]
    # one xy-plane per block needs Lx Ly = 32k; shared-memory tiles of 128 sites need
    # 128 % Lx == 0 and Ly % (128 / Lx) == 0
    dims = {5: (8, 4, 5, 3), 11: (16, 16, 2, 3)}.get(code, (6, 4, 5, 4))
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


@pytest.mark.parametrize("dims", [(16, 8, 3, 4), (8, 16, 2, 3), (32, 4, 2, 2), (4, 32, 2, 2)])
def test_hw_fp32_shared_tile_shapes(gpu_lib, dims):
    """The shared-memory tiled stencil when a tile is a whole xy-plane (its halo rows are
    its own rows), and for other row lengths (R = 128 / Lx rows per tile)."""
    import torch

    k = [i for i, v in enumerate(gpu_lib.hw32_variants()) if v[1] == 11][0]
    ctx, U = make_ctx(gpu_lib, dims, 0.6, 75)
    ctx.set_hw32_variant(k)
    nrhs = 3
    psi = S.gaussian_spinor(dims, 76, n=nrhs).astype(np.complex64)
    out = torch.empty(psi.shape, dtype=torch.complex64, device="cuda")
    ctx.apply_HW(to_dev(psi), out, nrhs, gpu_lib.OV_FP32)
    got = to_host(out).astype(np.complex128)
    for r in range(nrhs):
        assert rel(got[r], cimpl.hw_apply(U, psi[r].astype(np.complex128), M0)) < 3e-6


def test_hw_fp32_plane_variant_rejects_unfit_lattice(gpu_lib):
    """The plane-staged variant needs Lx Ly to be a multiple of 32 and the shared-memory
    tiled one 128 % Lx == 0: forced on another lattice they report OV_ERR_INVALID_ARG,
    and the autotuner skips them there."""
    import torch

    dims = (6, 4, 5, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.6, 73)
    psi = to_dev(S.gaussian_spinor(dims, 74, n=2).astype(np.complex64))
    out = torch.empty_like(psi)
    unfit = [i for i, v in enumerate(gpu_lib.hw32_variants()) if v[1] in (5, 11)]
    assert len(unfit) == 2
    for k in unfit:
        ctx.set_hw32_variant(k)
        with pytest.raises(gpu_lib.OvError) as e:
            ctx.apply_HW(psi, out, 2, gpu_lib.OV_FP32)
        assert e.value.code == gpu_lib.OV_ERR_INVALID_ARG
    ctx.set_hw32_variant(-1)
    ctx.apply_HW(psi, out, 2, gpu_lib.OV_FP32)
    want = wilson.apply_HW(U, to_host(psi).astype(np.complex128), M0)
    assert rel(to_host(out).astype(np.complex128), want) < 1e-5
