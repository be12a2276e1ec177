"""Pins for the oracle gradients of L = Re<eta, S_N b> (CPU only).

The link force is checked against central finite differences of L under
U_mu(x) -> exp(+-i h T_a) U_mu(x) and against the Daleckii-Krein formula for the
derivative of a matrix function; the source gradient against finite differences.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import contour, force, sign, wilson

DIMS = (2, 2, 2, 4)
M0 = 1.6


@pytest.fixture(scope="module")
def case():
    U = S.su3_links(DIMS, 0.4, 301)
    b = S.gaussian_spinor(DIMS, 302)
    eta = S.gaussian_spinor(DIMS, 303)
    z, c, c0 = contour.single_contour(16, 3.2, 3.2, 0.3)
    H = wilson.dense_HW(U, M0)
    y = sign.resolvents_dense(H, b.reshape(-1), z).reshape((16,) + b.shape)
    xi = sign.resolvents_dense(H, eta.reshape(-1), z.conj()).reshape((16,) + b.shape)
    F = force.link_force(U, y, xi, c)
    return U, b, eta, z, c, c0, F, H, y, xi


def _loss(U, b, eta, z, c, c0):
    s = sign.sign_apply_dense(wilson.dense_HW(U, M0), b.reshape(-1), z, c, c0)
    return np.vdot(eta.reshape(-1), s).real


def _rotate(U, mu, site, a, h):
    Up = U.copy()
    th = np.zeros(8)
    th[a] = h
    Up[(mu,) + site] = force.exp_generator(th) @ U[(mu,) + site]
    return Up


@pytest.mark.parametrize("mu,site,a", [(0, (0, 1, 0, 1), 0), (3, (3, 0, 1, 0), 7), (3, (1, 1, 1, 1), 4),
                                       (2, (2, 0, 0, 1), 2)])
def test_link_force_finite_difference(case, mu, site, a):
    U, b, eta, z, c, c0, F, *_ = case
    h = 1e-5
    fd = (_loss(_rotate(U, mu, site, a, h), b, eta, z, c, c0)
          - _loss(_rotate(U, mu, site, a, -h), b, eta, z, c, c0)) / (2 * h)
    assert abs(fd - F[(mu,) + site + (a,)]) < 1e-8 * max(1.0, abs(fd))


def test_link_force_daleckii_krein(case):
    """dS_N = V [Gamma o (V^dag dH V)] V^dag, Gamma_ik = (r(l_i) - r(l_k)) / (l_i - l_k)."""
    U, b, eta, z, c, c0, F, H, *_ = case
    lam, V = np.linalg.eigh(H)
    rl = contour.rational(lam, z, c, c0)
    dl = lam[:, None] - lam[None, :]
    same = np.abs(dl) < 1e-12
    rp = np.sum(c[None, :] / (z[None, :] - lam[:, None]) ** 2, axis=1)  # r'(lambda)
    G = np.where(same, rp[:, None] * np.ones_like(dl), (rl[:, None] - rl[None, :]) / np.where(same, 1, dl))
    mu, site, a = 1, (2, 1, 0, 1), 5
    T = force.su3_generators()[a]
    Ud = U.copy()
    Ud[(mu,) + site] = 1j * T @ U[(mu,) + site]
    Uz = U.copy()
    Uz[(mu,) + site] = 0
    dH = wilson.dense_HW(Ud, M0) - wilson.dense_HW(Uz, M0)  # H is affine in each link
    dS = V @ (G * (V.conj().T @ dH @ V)) @ V.conj().T
    dk = np.vdot(eta.reshape(-1), dS @ b.reshape(-1)).real
    assert abs(dk - F[(mu,) + site + (a,)]) < 1e-11 * max(1.0, abs(dk))


def test_source_gradient(case):
    U, b, eta, z, c, c0, F, H, y, xi = case
    g = force.source_gradient(xi, eta, c, c0)
    rng = np.random.default_rng(5)
    d = rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)
    h = 1e-6
    fd = (_loss(U, b + h * d, eta, z, c, c0) - _loss(U, b - h * d, eta, z, c, c0)) / (2 * h)
    assert abs(fd - np.vdot(g, d).real) < 1e-8 * max(1.0, abs(fd))
