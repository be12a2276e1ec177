"""Pins for the oracle's resolvent quadrature, sign function and overlap operator (CPU only)."""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl, contour, freefield, sign, wilson

DIMS = (2, 2, 2, 4)
M0 = 1.6


@pytest.fixture(scope="module")
def setup():
    U = S.su3_links(DIMS, 0.5, 101)
    H = wilson.dense_HW(U, M0)
    b = S.gaussian_spinor(DIMS, 102)
    return U, H, b


def test_quadrature_equals_rational_function_of_spectrum(setup):
    """(z - H)^-1 = sum_i v_i v_i^dag / (z - lambda_i) (the resolvent identity under Eq. 4)
    makes the per-node solve-and-sum exactly V r_N(Lambda) V^dag x."""
    U, H, b = setup
    z, c, c0 = contour.single_contour(32, 3.2, 3.2, 0.3)
    x = b.reshape(-1)
    s = sign.sign_apply_dense(H, x, z, c, c0)
    Sr, _ = sign.spectral_function(H, lambda l: contour.rational(l, z, c, c0))
    assert np.linalg.norm(s - Sr @ x) / np.linalg.norm(x) < 1e-13


def test_paper_contour_gives_spectral_sign(setup):
    """Eq. 5 with the paper's contours (500 nodes each) reproduces Eq. 2 to double precision.
    The paper's ellipses enclose |lambda| < 2.4, so H is scaled by 1/3 (sgn(cH) = sgn(H), c > 0)."""
    U, H, b = setup
    x = b.reshape(-1)
    lam = np.linalg.eigvalsh(H)
    assert np.abs(lam).max() / 3 < 2.3 and np.abs(lam).min() / 3 > 0.02
    z, c, c0 = contour.paper_two_contour(500)
    s = sign.sign_apply_dense(H / 3.0, x, z, c, c0)
    exact = sign.spectral_sign(H) @ x
    assert np.linalg.norm(s - exact) / np.linalg.norm(x) < 1e-13
    assert sign.sigma(x, s) < 1e-13


def test_cgnr_matches_dense(setup):
    U, H, b = setup
    z, c, c0 = contour.single_contour(8, 3.2, 3.2, 0.3)
    x = b.reshape(-1)
    yd = sign.resolvents_dense(H, x, z)
    for j in (0, 3):
        y, it, res = sign.cgnr_solve(U, b, z[j], M0, tol=1e-13)
        assert res < 2e-13
        assert np.linalg.norm(y.reshape(-1) - yd[j]) / np.linalg.norm(yd[j]) < 1e-11


def test_c_oracle_sign_matches_dense(setup):
    U, H, b = setup
    z, c, c0 = contour.single_contour(16, 3.2, 3.2, 0.3)
    s_dense = sign.sign_apply_dense(H, b.reshape(-1), z, c, c0)
    s_c, iters, res = cimpl.sign_apply(U, b, z, c, c0, M0, tol=1e-13)
    assert res.max() < 2e-13
    assert np.linalg.norm(s_c.reshape(-1) - s_dense) / np.linalg.norm(s_dense) < 1e-11


def test_free_field_closed_form():
    """At U = 1 the quadrature operator is r_N applied per momentum (FFT closed form)."""
    dims = (4, 4, 2, 4)
    U = S.unit_links(dims)
    b = S.gaussian_spinor(dims, 7)
    z, c, c0 = contour.single_contour(24, 3.3, 3.3, 0.3)
    got, _, _ = cimpl.sign_apply(U, b, z, c, c0, M0, tol=1e-13)
    want = freefield.apply_function(b, lambda e: contour.rational(e, z, c, c0), M0)
    assert np.linalg.norm(got - want) / np.linalg.norm(b) < 1e-11
    # and the exact free-field sign: sgn applied per momentum is an involution
    sg = freefield.apply_function(b, np.sign, M0)
    assert np.linalg.norm(freefield.apply_function(sg, np.sign, M0) - b) / np.linalg.norm(b) < 1e-13


def test_overlap_and_gw_identity(setup):
    """With D = (1 + gamma5 S)/2: {gamma5, D} - 2 D gamma5 D = gamma5 (1 - S^2) / 2 for any S."""
    U, H, b = setup
    z, c, c0 = contour.single_contour(12, 3.2, 3.2, 0.3)
    shp = b.shape
    Smat = sign.spectral_function(H, lambda l: contour.rational(l, z, c, c0))[0]

    def S_apply(v):
        return (Smat @ v.reshape(-1)).reshape(shp)

    def D0(v):
        return sign.overlap_from_sign(v, S_apply(v), 0.0)

    lhs = sign.gw_residual(D0, b)
    rhs = 0.5 * sign.g5(b - S_apply(S_apply(b)))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(b) < 1e-13
    # exact sign: GW holds to rounding
    Sx = sign.spectral_sign(H)

    def D0x(v):
        return sign.overlap_from_sign(v, (Sx @ v.reshape(-1)).reshape(shp), 0.0)

    assert np.linalg.norm(sign.gw_residual(D0x, b)) / np.linalg.norm(b) < 1e-13
    # Eq. 1 at m_q = 1 is the identity
    assert np.allclose(sign.overlap_from_sign(b, S_apply(b), 1.0), b)


def test_sign_gauge_covariant():
    dims = (2, 2, 2, 4)
    U = S.su3_links(dims, 0.6, 201)
    g = S.random_gauge_transform(dims, 202)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = np.einsum("...ab,...bc,...dc->...ad", g, U[mu], np.roll(g, -1, axis=-3 - mu).conj())
    b = S.gaussian_spinor(dims, 203)
    z, c, c0 = contour.single_contour(16, 3.2, 3.2, 0.3)
    s = sign.sign_apply_dense(wilson.dense_HW(U, M0), b.reshape(-1), z, c, c0).reshape(b.shape)
    gb = np.einsum("...ab,...sb->...sa", g, b)
    sg = sign.sign_apply_dense(wilson.dense_HW(Ug, M0), gb.reshape(-1), z, c, c0).reshape(b.shape)
    assert np.linalg.norm(sg - np.einsum("...ab,...sb->...sa", g, s)) / np.linalg.norm(b) < 1e-12


def test_c_oracle_many_sources_matches_dense(setup):
    """The batched C loop over (source, node) pairs gives, per source, the dense
    per-node solve-and-sum (Eqs. 5-7), and the non-strict single-source call reports an
    unconverged node instead of raising."""
    U, H, b = setup
    z, c, c0 = contour.single_contour(6, 3.2, 3.2, 0.3)
    B = np.stack([b, S.gaussian_spinor(DIMS, 103), S.point_sources(DIMS)[5]])
    got, iters, res = cimpl.sign_apply_many(U, B, z, c, c0, M0, tol=1e-13)
    assert iters.shape == (3, 6) and res.max() < 2e-13
    for k in range(3):
        want = sign.sign_apply_dense(H, B[k].reshape(-1), z, c, c0)
        assert np.abs(got[k].reshape(-1) - want).max() <= 1e-11 * np.abs(want).max()
    out, it, rr = cimpl.sign_apply(U, b, z, c, c0, M0, tol=1e-13, maxiter=3, strict=False)
    assert it.max() == 3 and rr.max() > 1e-6 and np.all(np.isfinite(out))
    with pytest.raises(RuntimeError):
        cimpl.sign_apply(U, b, z, c, c0, M0, tol=1e-13, maxiter=3)
