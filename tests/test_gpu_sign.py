"""sgn(H_W) b and D_ov(m_q) b on the GPU against the oracle, through the C ABI (GPU).

Parity: the GPU weighted sum of shifted-solver iterates vs the oracle's per-node
CGNR (or dense LU) resolvents and sum, same nodes, to 1e-10 relative.  Accuracy:
the same operator vs the exact spectral sign function (dense zheevd) within the
method error predicted from the spectrum.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl, contour, freefield, sign, wilson
from tests.gpu_common import M0, make_ctx, rel, rel_per_source, sgn_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu

PARITY = 1e-10


def _oracle(U, b, ctx, tol=1e-13):
    z, c, c0 = ctx.get_contour()
    out, iters, res = cimpl.sign_apply(U, b, z, c, c0, M0, tol=tol)
    return out


@pytest.mark.parametrize("mode", ["fp64", "fp64_2pass", "fp64_regen", "f32x2"])
def test_config1_4x4_dense(gpu_lib, mode):
    """4^4, eps = 0.3, N_q = 32 from Lanczos placement: parity with the per-node oracle,
    accuracy vs dense zheevd sgn, GW relation and sgn^2 = 1 within the predicted error."""
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, S.seed_for("config1"))
    spec = ctx.place_contour(32, steps=120)
    b = S.gaussian_spinor(dims, S.seed_for("config1.b"))
    got, st = sgn_gpu(ctx, b, tol=1e-12, mode=mode)
    assert st["converged"] == 1
    want = _oracle(U, b, ctx)
    assert rel(got, want) < PARITY
    # exact sign function and the method error predicted from the true spectrum
    H = wilson.dense_HW(U, M0)
    lam, V = np.linalg.eigh(H)
    z, c, c0 = ctx.get_contour()
    rl = contour.rational(lam, z, c, c0).real
    method_err = np.abs(rl - np.sign(lam)).max()
    assert abs(spec["lambda_max"] - lam.max()) < 1e-6 * lam.max()
    assert abs(spec["lambda_min"] - lam.min()) < 1e-6 * abs(lam.min())
    # the placement's prediction (from Lanczos bounds) matches the error on the true spectrum
    assert method_err <= 2.0 * spec["predicted_error"] + 1e-12
    assert spec["predicted_error"] < 1e-2
    x = b.reshape(-1)
    exact = (V * np.sign(lam)) @ (V.conj().T @ x)
    assert np.linalg.norm(got.reshape(-1) - exact) / np.linalg.norm(x) <= 1.01 * method_err + 1e-11
    # GW: {gamma5, D} - 2 D gamma5 D = gamma5 (1 - S^2)/2 at m_q = 0
    import torch

    Sb = to_dev(got)
    S2b = torch.empty_like(Sb)
    ctx.sgn(Sb, S2b, 1, ctx.opts(mode=mode))
    s2 = to_host(S2b)
    assert np.linalg.norm(s2 - b) / np.linalg.norm(b) <= 2.01 * method_err + 1e-10
    assert sign.sigma(b, got) <= 2.01 * method_err + 1e-10


@pytest.fixture(scope="module")
def config2(gpu_lib):
    """8^4, eps = 0.5, N_q = 64 (Lanczos placement), 4 Gaussian sources; the per-node CGNR
    oracle for all four (one solve per source and node, all pairs in parallel)."""
    dims = (8, 8, 8, 8)
    ctx, U = make_ctx(gpu_lib, dims, 0.5, S.seed_for("config2"))
    spec = ctx.place_contour(64, steps=150)
    b = S.gaussian_spinor(dims, S.seed_for("config2.b"), n=4)
    z, c, c0 = ctx.get_contour()
    want, _, _ = cimpl.sign_apply_many(U, b, z, c, c0, M0, tol=1e-13)
    return ctx, U, b, spec, want


@pytest.mark.parametrize("mode", ["fp64", "fp64_2pass", "fp64_regen", "f32x2"])
def test_config2_8x4_parity(gpu_lib, config2, mode):
    """tol 1e-12, 4 sources in one call; every source against the per-node CGNR oracle at
    1e-10 (element-wise and in norm), and sgn^2 b = b within the predicted method error."""
    import torch

    ctx, U, b, spec, want = config2
    got, st = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode=mode)
    assert st["converged"] == 1 and st["max_residual"] <= 1e-12
    errs = rel_per_source(got, want)
    assert max(errs) < PARITY, errs
    S2 = torch.empty_like(to_dev(got))
    ctx.sgn(to_dev(got), S2, 4, ctx.opts(mode=mode))
    s2 = to_host(S2)
    for k in range(4):
        assert rel(s2[k], b[k]) < max(10 * spec["predicted_error"], 1e-9)


@pytest.mark.parametrize("mode", ["fp64_2pass", "fp64_regen", "f32x2"])
def test_two_pass_equals_shifted(gpu_lib, config2, mode):
    """The coefficient-space forms (stored basis, regenerated basis) and the vector-space
    shifted form compute the same Galerkin iterates: agreement to rounding, per source."""
    ctx, U, b, spec, want = config2
    a, sa = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode="fp64")
    c, sc = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode=mode)
    # the reductions are grouped differently, so alpha/beta differ in the last bits and the
    # stopping iteration near tol = 1e-12 moves by a few percent; the results agree to
    # the solver accuracy
    assert abs(sa["iterations"] - sc["iterations"]) <= 0.15 * sa["iterations"]
    for k in range(4):
        assert rel(c[k], a[k]) < 1e-11
    assert sc["node_updates"] == 0 and sa["node_updates"] > 0


@pytest.mark.parametrize("groups", [0, 1], ids=["auto-groups", "one-launch"])
@pytest.mark.parametrize("mode", ["fp64", "fp64_2pass", "fp64_regen", "f32x2"])
def test_ragged_lattice_parity(gpu_lib, mode, groups):
    """Lattice whose volume is not a multiple of any block size; 3 sources, either one
    graph branch per source or all three in each launch (the stencil grid then holds the
    three sources of every 32-site tile side by side, the last tile ragged)."""
    dims = (3, 5, 4, 6)
    ctx, U = make_ctx(gpu_lib, dims, 0.5, 51)
    ctx.set_concurrency(groups)
    ctx.set_contour_ellipse(24, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 52, n=3)
    got, st = sgn_gpu(ctx, b, tol=1e-12, mode=mode)
    for k in range(3):
        assert rel(got[k], _oracle(U, b[k], ctx)) < PARITY


def test_free_field_closed_form_8x4(gpu_lib):
    dims = (8, 8, 8, 8)
    ctx, _ = make_ctx(gpu_lib, dims, 0.0, 0)
    ctx.set_contour_ellipse(48, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 61)
    got, st = sgn_gpu(ctx, b, tol=1e-13)
    z, c, c0 = ctx.get_contour()
    want = freefield.apply_function(b, lambda e: contour.rational(e, z, c, c0), M0)
    assert rel(got, want) < PARITY


def test_paper_two_contour_form(gpu_lib):
    """Eq. 5 form (two ellipses, c0 = 0) with the paper's alpha = 0.1, scaled to enclose the spectrum."""
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 71)
    ctx.set_contour_ellipse(48, 3.4, 3.39999, 0.1, gpu_lib.OV_CONTOUR_PAIR)
    z, c, c0 = ctx.get_contour()
    zr, cr, c0r = contour.paper_two_contour(48, 3.4, 3.39999, 0.1)
    assert np.allclose(z, zr, rtol=0, atol=1e-14) and np.allclose(c, cr, rtol=0, atol=1e-15) and c0 == c0r
    b = S.gaussian_spinor(dims, 72)
    got, st = sgn_gpu(ctx, b, tol=1e-12)
    assert rel(got, _oracle(U, b, ctx)) < PARITY


def test_overlap_epilogue(gpu_lib):
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 81)
    ctx.set_contour_ellipse(32, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 82)
    s, _ = sgn_gpu(ctx, b)
    out = torch.empty_like(to_dev(b))
    ctx.overlap(0.1, to_dev(b), out, 1)
    want = sign.overlap_from_sign(b, _oracle(U, b, ctx), 0.1)
    assert rel(to_host(out), want) < PARITY


def test_host_io_matches_device_io(gpu_lib):
    """Host buffers, pageable (copied by the copy engine) and page-locked (read by a
    kernel), give the device-buffer result bit for bit, for the sign and the overlap."""
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 91)
    ctx.set_contour_ellipse(32, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 92, n=2)
    dev, _ = sgn_gpu(ctx, b, nrhs=2)
    out = np.empty_like(b)
    ctx.sgn(b, out, 2, ctx.opts(host_io=True))
    assert np.array_equal(out, dev)
    hb = torch.from_numpy(b).pin_memory()
    ho = torch.empty_like(hb).pin_memory()
    ctx.sgn(hb, ho, 2, ctx.opts(host_io=True))
    assert np.array_equal(ho.numpy(), dev)
    bd = to_dev(b)
    od = torch.empty_like(bd)
    ctx.overlap(0.1, bd, od, 2, ctx.opts())
    ctx.overlap(0.1, hb, ho, 2, ctx.opts(host_io=True))
    assert np.array_equal(ho.numpy(), to_host(od))


def test_graph_and_direct_launch_agree_bitwise(gpu_lib):
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 93)
    ctx.set_contour_ellipse(32, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 94, n=2)
    a1, _ = sgn_gpu(ctx, b, use_graph=True)
    a2, _ = sgn_gpu(ctx, b, use_graph=False, check_every=7)
    assert np.array_equal(a1, a2)


@pytest.mark.parametrize("mode", ["fp64", "fp64_2pass", "fp64_regen", "f32x2"])
def test_edge_cases(gpu_lib, mode):
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 95)
    ctx.set_contour_ellipse(16, 3.4, 3.4, 0.3)
    # zero source -> zero output
    z0, st = sgn_gpu(ctx, np.zeros(S.lattice_shape(dims) + (4, 3), np.complex128), mode=mode)
    assert np.all(z0 == 0) and st["converged"] == 1
    # iteration cap -> NOT_CONVERGED, output holds the current iterate
    b = S.gaussian_spinor(dims, 96)
    bd = to_dev(b)
    out = torch.empty_like(bd)
    st = ctx.sgn(bd, out, 1, ctx.opts(max_iter=3, mode=mode), allow_not_converged=True)
    assert st["status"] == gpu_lib.OV_ERR_NOT_CONVERGED and st["converged"] == 0
    # NaN in the source -> BREAKDOWN status, no hang
    bn = b.copy()
    bn[0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(gpu_lib.OvError) as e:
        sgn_gpu(ctx, bn, mode=mode)
    assert e.value.code == gpu_lib.OV_ERR_BREAKDOWN
    # a zero source next to a nonzero one in the same call
    bz = np.stack([np.zeros_like(b), b])
    mixed, _ = sgn_gpu(ctx, bz, nrhs=2, mode=mode)
    alone, _ = sgn_gpu(ctx, b, mode=mode)
    assert np.all(mixed[0] == 0) and np.array_equal(mixed[1], alone)
    # nrhs = 0 is a no-op
    ctx.sgn(bd, out, 0)
    # bad options
    with pytest.raises(gpu_lib.OvError):
        ctx.sgn(bd, out, 1, ctx.opts(tol=0.0))
    # no contour
    ctx2 = gpu_lib.Context(dims)
    ctx2.set_gauge(to_dev(U))
    with pytest.raises(gpu_lib.OvError) as e:
        ctx2.sgn(bd, out, 1)
    assert e.value.code == gpu_lib.OV_ERR_NO_CONTOUR


def test_persistent_and_per_iteration_launches_agree(gpu_lib, config2):
    """The cooperative persistent loop and the per-iteration (graph) kernels run the same
    recurrences (partial sums grouped differently): results agree to solver accuracy."""
    ctx, U, b, spec, want = config2
    ctx.set_persistent(True)
    a, sa = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode="fp64_2pass")
    ctx.set_persistent(False)
    c, sc = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode="fp64_2pass")
    assert abs(sa["iterations"] - sc["iterations"]) <= 0.15 * sc["iterations"]
    assert sa["launches"] < sc["launches"]
    for k in range(4):
        assert rel(a[k], c[k]) < 1e-11
    assert max(rel_per_source(a, want)) < 1e-10


@pytest.mark.parametrize("mode", ["fp64", "fp64_2pass", "fp64_regen", "f32x2"])
def test_source_groups_give_identical_results(gpu_lib, config2, mode):
    """Replaying the per-iteration kernels as 1, 2 or 4 parallel graph branches over the
    sources changes no arithmetic: bitwise identical results and iteration counts."""
    ctx, U, b, spec, want = config2
    outs = []
    for groups in (1, 2, 4):
        ctx.set_concurrency(groups)
        outs.append(sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode=mode))
    ctx.set_concurrency(0)
    for o, st in outs[1:]:
        assert np.array_equal(o, outs[0][0]) and st["iterations"] == outs[0][1]["iterations"]


def test_zolotarev_nodes_4x4(gpu_lib):
    """Zolotarev node set (16 pole pairs) placed from Lanczos bounds on 4^4: parity with the
    per-node oracle on the same nodes, and the exact sign function (dense zheevd) within
    the predicted error, far below the 32-node ellipse's."""
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, S.seed_for("config1"))
    spec = ctx.place_zolotarev(16, steps=120)
    b = S.gaussian_spinor(dims, S.seed_for("config1.b"))
    got, st = sgn_gpu(ctx, b, tol=1e-13, mode="fp64_2pass")
    assert rel(got, _oracle(U, b, ctx)) < PARITY
    lam, V = np.linalg.eigh(wilson.dense_HW(U, M0))
    assert spec["gap"] <= np.abs(lam).min() and spec["abs_max_bound"] >= np.abs(lam).max()
    assert spec["predicted_error"] < 1e-12
    exact = (V * np.sign(lam)) @ (V.conj().T @ b.reshape(-1))
    assert np.linalg.norm(got.reshape(-1) - exact) / np.linalg.norm(b) <= 1e-11


@pytest.mark.parametrize("mode", ["fp64_2pass", "f32x2"])
def test_zolotarev_nodes_8x4_sign_squared(gpu_lib, config2, mode):
    """8^4 config-2 links with 16 Zolotarev pole pairs: sgn^2 b = b to 1e-10 (the 64-node
    ellipse reaches only its ~1e-8 method error); the ellipse is restored afterwards."""
    import torch

    ctx, U, b, spec, want = config2
    z, c, c0 = ctx.get_contour()
    try:
        zs = ctx.place_zolotarev(16, steps=150)
        assert zs["predicted_error"] < 1e-11
        got, st = sgn_gpu(ctx, b, nrhs=4, tol=1e-13, mode=mode)
        S2 = torch.empty_like(to_dev(got))
        ctx.sgn(to_dev(got), S2, 4, ctx.opts(mode=mode, tol=1e-13))
        s2 = to_host(S2)
        for k in range(4):
            assert rel(s2[k], b[k]) < 1e-10
    finally:
        ctx.set_contour(z, c, c0)


@pytest.mark.parametrize("mode", ["fp64_2pass", "f32x2"])
def test_store_depth_changes_reuse_no_stale_graph(gpu_lib, config2, mode):
    """Calls with different stored-basis depths (max_iter, and the depth learned from the
    previous call) on one context give the results of a fresh context: graphs captured for
    one depth are not replayed for another."""
    ctx, U, b, spec, want = config2
    a1, _ = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode=mode, max_iter=2000)
    a2, _ = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode=mode, max_iter=600)
    a3, _ = sgn_gpu(ctx, b, nrhs=4, tol=1e-12, mode=mode)
    fresh, _ = make_ctx(gpu_lib, (8, 8, 8, 8), 0.5, S.seed_for("config2"))
    z, c, c0 = ctx.get_contour()
    fresh.set_contour(z, c, c0)
    want, _ = sgn_gpu(fresh, b, nrhs=4, tol=1e-12, mode=mode, max_iter=2000)
    for got in (a1, a2, a3):
        assert np.all(np.isfinite(got))
        for k in range(4):
            assert rel(got[k], want[k]) < 1e-13


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (1, 2, 3, 4), (5, 1, 1, 3)])
@pytest.mark.parametrize("mode", ["fp64", "fp64_2pass", "f32x2"])
def test_degenerate_lattices(gpu_lib, dims, mode):
    """Extents 1 and 2, where a site is its own neighbour or both neighbours coincide:
    parity with the oracle (which builds the hops with periodic rolls)."""
    ctx, U = make_ctx(gpu_lib, dims, 0.5, 57)
    ctx.set_contour_ellipse(24, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 58, n=2)
    got, st = sgn_gpu(ctx, b, tol=1e-12, mode=mode)
    for k in range(2):
        assert rel(got[k], _oracle(U, b[k], ctx)) < PARITY


def test_many_sources_one_call(gpu_lib):
    """40 sources in one call (more than any graph-branch or batch count): each equals
    its solve alone."""
    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 61)
    ctx.set_contour_ellipse(16, 3.4, 3.4, 0.3)
    b = S.gaussian_spinor(dims, 62, n=40)
    for mode in ("fp64_2pass", "f32x2"):
        allb, st = sgn_gpu(ctx, b, nrhs=40, tol=1e-12, mode=mode)
        for k in (0, 17, 39):
            one, _ = sgn_gpu(ctx, b[k], tol=1e-12, mode=mode)
            assert rel(allb[k], one) < 1e-12


def test_empty_contour_is_c0_times_b(gpu_lib):
    """A quadrature with no nodes (a rank of a node-sharded sum that holds none) is
    S_N = c0: the library returns c0 b, and D_ov follows from it (Eq. 1)."""
    import torch

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(gpu_lib, dims, 0.3, 97)
    c0 = 0.7 - 0.2j
    ctx.set_contour(np.zeros(0, np.complex128), np.zeros(0, np.complex128), c0)
    z, c, cc0 = ctx.get_contour()
    assert len(z) == 0 and cc0 == c0
    b = S.gaussian_spinor(dims, 98, n=2)
    for mode in ("fp64", "fp64_2pass", "f32x2", "mixed"):
        got, st = sgn_gpu(ctx, b, tol=1e-12, mode=mode)
        assert st["converged"] == 1 and st["iterations"] == 0
        assert rel(got, c0 * b) <= 1e-15
    out = torch.empty_like(to_dev(b))
    ctx.overlap(0.1, to_dev(b), out, 2)
    assert rel(to_host(out), sign.overlap_from_sign(b, c0 * b, 0.1)) < 1e-15


@pytest.mark.parametrize("mode", ["fp64_2pass", "f32x2", "fp64"])
def test_node_list_not_closed_under_conjugation(gpu_lib, mode):
    """A node list without conjugate partners gives complex Lanczos-basis coefficients
    (the stored-basis sum then takes its complex form); parity with the oracle."""
    dims = (4, 4, 4, 8)
    ctx, U = make_ctx(gpu_lib, dims, 0.4, 1501)
    z = np.array([1.0 + 1.5j, -2.0 + 0.8j, 4.0 - 1.2j])
    c = np.array([0.5 - 0.2j, -0.3 + 0.7j, 0.25 + 0.1j])
    ctx.set_contour(z, c, 0.3 + 0.4j)
    b = S.gaussian_spinor(dims, 1502, n=2)
    got, st = sgn_gpu(ctx, b, tol=1e-12, mode=mode)
    want, _, _ = cimpl.sign_apply_many(U, b, z, c, 0.3 + 0.4j, M0, tol=1e-13)
    assert max(rel_per_source(got, want)) < PARITY
