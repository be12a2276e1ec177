"""Hermitian Wilson-Dirac operator H_W = gamma5 D_W(-m0) (oracle; test infrastructure only).

The paper introduces H_W right after Eq. 1 as gamma5 times the Wilson-Dirac
operator at negative mass -m0, with the standard (Wilson-kernel) overlap setup
of Sec. "Numerical experiments".  It does not write D_W out; we take the standard
normalisation

    (H_W psi)(x) = gamma5 [ (4 r + m) psi(x)
                            - 1/2 sum_mu ( (r - gamma_mu) U_mu(x) psi(x + mu)
                                         + (r + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ) ],
    m = -m0,

periodic in x, y, z and periodic (bc_t = +1) or antiperiodic (bc_t = -1) in t,
the sign applied to every hop that crosses the t boundary.

Arrays use the canonical layouts documented in ``synthetic``: U has shape
(4, Lt, Lz, Ly, Lx, 3, 3); spinors have shape (..., Lt, Lz, Ly, Lx, 4, 3).
"""
from __future__ import annotations

import numpy as np

from .gamma import gamma5, gamma_matrices


def _spin(mat, psi):
    return np.einsum("st,...tc->...sc", mat, psi)


def _shift(psi, mu, step, bc_t):
    """psi(x + step * mu-hat) with the boundary sign on hops across t."""
    ax = -3 - mu
    out = np.roll(psi, -step, axis=ax)
    if mu == 3 and bc_t != 1.0:
        lt = psi.shape[ax]
        if step == +1:
            out[..., lt - 1, :, :, :, :, :] *= bc_t
        else:
            out[..., 0, :, :, :, :, :] *= bc_t
    return out


def apply_DW(U, psi, m0, r=1.0, bc_t=-1.0):
    """D_W(-m0) psi for a batch of spinors (the bracket in the formula above)."""
    psi = np.asarray(psi, dtype=np.complex128)
    g = gamma_matrices()
    eye = np.eye(4, dtype=np.complex128)
    out = (4.0 * r - m0) * psi
    for mu in range(4):
        ax = -3 - mu
        fwd = _shift(psi, mu, +1, bc_t)
        bwd = _shift(psi, mu, -1, bc_t)
        U_here = U[mu]
        U_back = np.roll(U[mu], +1, axis=ax)  # U_mu(x - mu)
        hop_f = np.einsum("...ab,...sb->...sa", U_here, fwd)
        hop_b = np.einsum("...ba,...sb->...sa", U_back.conj(), bwd)
        out = out - 0.5 * (_spin(r * eye - g[mu], hop_f) + _spin(r * eye + g[mu], hop_b))
    return out


def apply_HW(U, psi, m0, r=1.0, bc_t=-1.0):
    """H_W psi = gamma5 D_W(-m0) psi (Eq. 1 context)."""
    return _spin(gamma5(), apply_DW(U, psi, m0, r, bc_t))


def dense_HW(U, m0, r=1.0, bc_t=-1.0, chunk=256):
    """H_W as a dense (12V x 12V) complex matrix, built column by column.

    Row/column index = ((((t*Lz + z)*Ly + y)*Lx + x)*4 + spin)*3 + colour,
    i.e. the flattened canonical spinor layout."""
    shp = U.shape[1:5]
    n = int(np.prod(shp)) * 12
    H = np.empty((n, n), dtype=np.complex128)
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        E = np.zeros((j1 - j0, n), dtype=np.complex128)
        E[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
        cols = apply_HW(U, E.reshape((j1 - j0,) + shp + (4, 3)), m0, r, bc_t)
        H[:, j0:j1] = cols.reshape(j1 - j0, n).T
    return H
