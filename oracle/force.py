"""Gradients of L = Re<eta, S_N b> (oracle; test infrastructure only).

S_N = c0 + sum_j c_j (z_j - H)^-1 is the quadrature of Eqs. 4-7.  Differentiating
each resolvent, d(z - H)^-1 = (z - H)^-1 dH (z - H)^-1, gives

    dL = Re sum_j c_j xi_j^dag dH y_j,   y_j = (z_j - H)^-1 b,   xi_j = (conj(z_j) - H)^-1 eta,

and with respect to the source, dL = Re<g_b, db> with g_b = S_N^dag eta
= conj(c0) eta + sum_j conj(c_j) xi_j.

Link variation: U_mu(x) -> exp(i omega_a T_a) U_mu(x), T_a = lambda_a / 2 (Gell-Mann).
U_mu(x) enters H_W twice: in the forward hop at x and (as U^dag) in the backward
hop at x + mu.  Writing Gamma_1 = gamma5 (r - gamma_mu), Gamma_2 = gamma5 (r + gamma_mu)
and s = -1 on links that cross the antiperiodic t boundary (else +1),

    dL/d omega_a = 1/2 Im tr[ T_a M ],
    M = s * sum_j c_j ( sum_spin [Gamma_1 U y_j(x+mu)] (x) xi_j(x)^*
                      - sum_spin [Gamma_2 y_j(x)] (x) [U xi_j(x+mu)]^* ),

where (x) is the colour outer product (row index from the left factor).
"""
from __future__ import annotations

import numpy as np

from .gamma import gamma5, gamma_matrices
from .wilson import _shift, _spin


def su3_generators() -> np.ndarray:
    """T_a = lambda_a / 2, a = 1..8, as an array (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam / 2


def link_force(U, y, xi, c, r=1.0, bc_t=-1.0):
    """dL/d omega_{x,mu,a} as an array (4, Lt, Lz, Ly, Lx, 8).

    y, xi: arrays (N, Lt, Lz, Ly, Lx, 4, 3) of forward and adjoint resolvents;
    c: the N quadrature coefficients."""
    g = gamma_matrices()
    g5m = gamma5()
    eye = np.eye(4)
    T = su3_generators()
    c = np.asarray(c, dtype=np.complex128)
    F = np.zeros((4,) + U.shape[1:5] + (8,))
    for mu in range(4):
        G1 = g5m @ (r * eye - g[mu])
        G2 = g5m @ (r * eye + g[mu])
        yf = _shift(y, mu, +1, bc_t)   # y(x + mu), boundary sign included
        xf = _shift(xi, mu, +1, bc_t)  # xi(x + mu), boundary sign included
        A1 = _spin(G1, np.einsum("...ab,...sb->...sa", U[mu], yf))
        M1 = np.einsum("j,j...sb,j...sa->...ba", c, A1, xi.conj())
        A2 = _spin(G2, y)
        Uxf = np.einsum("...ab,...sb->...sa", U[mu], xf)
        M2 = np.einsum("j,j...sb,j...sg->...bg", c, A2, Uxf.conj())
        M = M1 - M2
        F[mu] = 0.5 * np.einsum("aij,...ji->...a", T, M).imag
    return F


def source_gradient(xi, eta, c, c0):
    """g_b = S_N^dag eta = conj(c0) eta + sum_j conj(c_j) xi_j."""
    return np.conj(c0) * eta + np.tensordot(np.conj(c), xi, axes=(0, 0))


def exp_generator(theta8: np.ndarray) -> np.ndarray:
    """exp(i sum_a theta_a T_a) for theta8[..., 8], by eigendecomposition."""
    X = np.einsum("...a,aij->...ij", theta8, su3_generators())
    w, V = np.linalg.eigh(X)
    return np.einsum("...ik,...k,...jk->...ij", V, np.exp(1j * w), V.conj())
