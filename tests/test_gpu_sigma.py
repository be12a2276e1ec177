"""Quality of the sign function versus the number of nodes with the paper's contour form
(two ellipses, alpha = 0.1, rho = 1.1999, centres +-1.2; integration setup of the
Supplement), rescaled by the Lanczos bound of |lambda|: sigma = |s's - b'b| / b'b falls
with N and reaches double precision by N = 500 per contour, the behaviour the paper
reports for its ensemble (Sec. "Results")."""
import numpy as np
import pytest

import synthetic as S
from oracle import sign, wilson
from tests.gpu_common import M0, make_ctx, sgn_gpu

pytestmark = pytest.mark.gpu


def test_sigma_vs_nodes_paper_contour(gpu_lib):
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, S.seed_for("sigma"))
    spec = ctx.place_contour(16, steps=120)
    scale = spec["abs_max_bound"] / 2.35  # spectrum / scale inside (0.0001, 2.3999)
    b = S.gaussian_spinor(dims, S.seed_for("sigma.b"))
    H = wilson.dense_HW(U, M0)
    exact = sign.spectral_sign(H) @ b.reshape(-1)
    sig, err = {}, {}
    for n in (100, 250, 500, 1000):
        ctx.set_contour_ellipse(n, 1.2 * scale, 1.1999 * scale, 0.1, gpu_lib.OV_CONTOUR_PAIR)
        s, st = sgn_gpu(ctx, b, tol=1e-13, mode="fp64_2pass")
        assert st["converged"] == 1
        sig[n] = sign.sigma(b, s)
        err[n] = np.linalg.norm(s.reshape(-1) - exact) / np.linalg.norm(b)
    assert sig[100] > sig[500]
    assert sig[500] < 1e-12 and sig[1000] < 1e-12
    assert err[1000] < 1e-11
