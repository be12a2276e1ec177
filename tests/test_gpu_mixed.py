"""Mixed-precision solves against the FP64 forms and the oracle, through the C ABI (GPU):
"mixed" (FP32 Lanczos + FP64 true residuals + batched FP32 corrections) and "f32x2"
(double-float vector arithmetic, FP64 scalars and sum)."""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl
from tests.gpu_common import M0, make_ctx, rel, sgn_gpu

pytestmark = pytest.mark.gpu


def test_mixed_small_matches_fp64_and_oracle(gpu_lib):
    dims = (6, 6, 6, 8)
    ctx, U = make_ctx(gpu_lib, dims, 0.5, 501)
    ctx.place_contour(32, steps=120)
    b = S.gaussian_spinor(dims, 502, n=3)
    mx, sm = sgn_gpu(ctx, b, nrhs=3, tol=1e-12, mode="mixed")
    fp, sf = sgn_gpu(ctx, b, nrhs=3, tol=1e-12, mode="fp64_2pass")
    assert sm["converged"] == 1 and sm["max_residual"] <= 1e-12
    assert sm["refine_rounds"] >= 1
    for k in range(3):
        assert rel(mx[k], fp[k]) < 1e-10
    z, c, c0 = ctx.get_contour()
    want, _, _ = cimpl.sign_apply(U, b[0], z, c, c0, M0, tol=1e-13)
    assert rel(mx[0], want) < 1e-10


@pytest.fixture(scope="module", params=[((16, 16, 16, 16), 0.5, 64), ((16, 16, 16, 32), 0.6, 64)],
                ids=["16^4", "16^3x32"])
def full_size(gpu_lib, request):
    """16^4 (eps 0.5) and 16^3 x 32 (eps 0.6), N_q = 64, the 12 spin-colour point sources,
    and the plain FP64 GPU result (two-pass form) they are checked against."""
    dims, eps, nq = request.param
    ctx, U = make_ctx(gpu_lib, dims, eps, S.seed_for("gauge:" + "x".join(map(str, dims))))
    ctx.place_contour(nq, steps=150)
    b = S.point_sources(dims)
    fp, sf = sgn_gpu(ctx, b, nrhs=12, tol=1e-12, mode="fp64_2pass")
    assert sf["converged"] == 1
    return ctx, b, fp


@pytest.mark.parametrize("mode", ["mixed", "f32x2"])
def test_mixed_full_size_point_sources(gpu_lib, full_size, mode):
    """All 12 right-hand sides in one call; error vs the plain FP64 GPU form <= 1e-10 per source."""
    ctx, b, fp = full_size
    mx, sm = sgn_gpu(ctx, b, nrhs=12, tol=1e-12, mode=mode)
    assert sm["converged"] == 1
    errs = [rel(mx[k], fp[k]) for k in range(12)]
    assert max(errs) < 1e-10, errs


@pytest.mark.parametrize("mode", ["mixed", "f32x2"])
def test_mixed_edge_cases(gpu_lib, mode):
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 511)
    ctx.set_contour_ellipse(16, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 512)
    bz = np.stack([np.zeros_like(b), b])
    out, st = sgn_gpu(ctx, bz, nrhs=2, mode=mode)
    assert np.all(out[0] == 0)
    fp, _ = sgn_gpu(ctx, b, mode="fp64")
    assert rel(out[1], fp) < 1e-10
