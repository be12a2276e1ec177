"""Full-size parity: the benchmark's lattices against the CPU oracle, through the C ABI (GPU).

16^4 (eps 0.5) and 16^3 x 32 (eps 0.6) with the 12 spin-colour point sources in ONE call,
in the coefficient-space FP64 form and the double-float form.  At these sizes the solver
takes paths it never takes on small lattices: stencil grids of many waves, and the stored
Lanczos basis solved in batches of sources that fit the device (a fresh context starts
with a deep store, so the 12 sources split into several batches).

The oracle (per-node CGNR, Eq. 6, then the weighted sum of Eqs. 5-7) runs on the host
cores, so the contour is short: two conjugate pairs of nodes with |Im z| >= 1.5 (a valid
quadrature S_N = c0 + sum_j c_j (z_j - H)^-1 for parity, not an approximation of sgn).
Checked against the oracle, element by element and in norm, to 1e-10:
  * source 0 and source 7 on their own;
  * a seeded random combination sum_k a_k b_k of all 12 sources (S_N is linear, so every
    source's output enters the comparison with a nonzero weight).
And on all 12 outputs: the 12 x 12 block of S_N at the source site is hermitian.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl
from tests.gpu_common import M0, make_ctx, rel, sgn_gpu

pytestmark = pytest.mark.gpu

PARITY = 1e-10
# two conjugate pairs (S_N hermitian), far enough from the real axis for a short CGNR
Z = np.array([1.0 + 1.5j, 4.5 + 1.8j, 4.5 - 1.8j, 1.0 - 1.5j])
C = np.array([0.7 - 0.2j, -0.4 + 0.9j, -0.4 - 0.9j, 0.7 + 0.2j])
C0 = -1.0 + 0.0j
SINGLE = (0, 7)


@pytest.fixture(scope="module", params=[((16, 16, 16, 16), 0.5), ((16, 16, 16, 32), 0.6)],
                ids=["16^4", "16^3x32"])
def full(gpu_lib, request):
    dims, eps = request.param
    U = S.su3_links(dims, eps, S.seed_for("gauge:" + "x".join(map(str, dims))))
    b = S.point_sources(dims)
    rng = np.random.default_rng(S.seed_for("fullsize.mix"))
    a = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    mix = np.tensordot(a, b, axes=(0, 0))
    srcs = np.stack([b[k] for k in SINGLE] + [mix])
    want, iters, res = cimpl.sign_apply_many(U, srcs, Z, C, C0, M0, tol=1e-13)
    assert res.max() < 1e-12
    return dims, U, b, a, want


@pytest.mark.parametrize("mode", ["fp64_2pass", "f32x2"])
def test_point_sources_full_size_vs_oracle(gpu_lib, full, mode):
    import torch

    dims, U, b, a, want = full
    ctx = gpu_lib.Context(dims, bc_t=-1, m0=M0)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    ctx.set_contour(Z, C, C0)
    got, st = sgn_gpu(ctx, b, nrhs=12, tol=1e-12, mode=mode)
    assert st["converged"] == 1 and st["max_residual"] <= 1e-12
    for i, k in enumerate(SINGLE):
        assert rel(got[k], want[i]) < PARITY, (k, rel(got[k], want[i]))
    combo = np.tensordot(a, got, axes=(0, 0))
    assert rel(combo, want[-1]) < PARITY, rel(combo, want[-1])
    # all 12: the block <e_k, S_N e_l> at the source site (the origin) is hermitian
    G = got[:, 0, 0, 0, 0].reshape(12, 12).T
    assert np.abs(G - G.conj().T).max() <= 1e-12 * np.abs(G).max()
    ctx.close()
