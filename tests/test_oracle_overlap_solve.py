"""Pins of the oracle's overlap solve x = D_ov(m_q)^-1 b (Eq. 1 with the quadrature sign).

The dense LU solve is checked against the free-field momentum-space inverse (an
independent closed form), against m_q = 1 (D = 1), against gamma5-hermiticity of D, and
-- with the exact sign function -- against the Ginsparg-Wilson identity of the inverse,
gamma5 D^-1 + D^-1 gamma5 = 2 gamma5 at m_q = 0."""
import numpy as np
import pytest

import synthetic as S
from oracle import contour, freefield, sign, wilson

M0 = 1.6


def _flat(x):
    return np.asarray(x).reshape(-1)


@pytest.mark.parametrize("m_q", [0.05, 0.3])
def test_free_field_dense_solve_matches_momentum_inverse(m_q):
    dims = (4, 4, 4, 4)
    U = S.unit_links(dims)
    H = wilson.dense_HW(U, M0)
    z, c, c0 = contour.single_contour(32, 3.3, 3.3, 0.3)
    b = S.gaussian_spinor(dims, 701)
    x = sign.overlap_solve_dense(H, b, z, c, c0, m_q)
    rN = lambda e: contour.rational(e, z, c, c0)
    want = freefield.overlap_inverse(b, rN, m_q, M0)
    assert np.linalg.norm(x - _flat(want)) <= 1e-12 * np.linalg.norm(want)


def test_dense_operator_is_gamma5_hermitian_and_solves():
    dims = (2, 2, 2, 4)
    U = S.su3_links(dims, 0.5, 702)
    H = wilson.dense_HW(U, M0)
    z, c, c0 = contour.single_contour(24, 3.4, 3.4, 0.3)
    D = sign.overlap_dense(H, z, c, c0, 0.1)
    g = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), D.shape[0] // 12)
    assert np.abs(D.conj().T - g[:, None] * D * g[None, :]).max() <= 1e-13
    b = S.gaussian_spinor(dims, 703)
    x = sign.overlap_solve_dense(H, b, z, c, c0, 0.1)
    assert np.linalg.norm(D @ x - _flat(b)) <= 1e-13 * np.linalg.norm(b)
    # D_ov(1) = 1
    x1 = sign.overlap_solve_dense(H, b, z, c, c0, 1.0)
    assert np.linalg.norm(x1 - _flat(b)) <= 1e-14 * np.linalg.norm(b)


def test_inverse_satisfies_ginsparg_wilson_with_exact_sign():
    """With S = sgn(H) (S^2 = 1), {gamma5, D(0)} = 2 D gamma5 D, so gamma5 D^-1 + D^-1 gamma5 = 2 gamma5."""
    dims = (2, 2, 2, 4)
    U = S.su3_links(dims, 0.5, 704)
    H = wilson.dense_HW(U, M0)
    n = H.shape[0]
    Sx = sign.spectral_sign(H)
    g = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), n // 12)
    D = 0.5 * np.eye(n) + 0.5 * g[:, None] * Sx
    Dinv = np.linalg.inv(D)
    G = np.diag(g)
    assert np.abs(G @ Dinv + Dinv @ G - 2 * G).max() <= 1e-11
    # the quadrature operator reproduces it within its method error
    z, c, c0 = contour.single_contour(64, 3.4, 3.4, 0.3)
    lam = np.linalg.eigvalsh(H)
    err = np.abs(contour.rational(lam, z, c, c0).real - np.sign(lam)).max()
    Dq = sign.overlap_dense(H, z, c, c0, 0.0)
    Dqinv = np.linalg.inv(Dq)
    assert np.abs(G @ Dqinv + Dqinv @ G - 2 * G).max() <= 1e3 * err + 1e-11
