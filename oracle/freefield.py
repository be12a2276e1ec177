"""Free-field (U = 1) closed form in momentum space (oracle; test infrastructure only).

With all links equal to 1 a plane wave exp(i p.x) u is an eigenvector of the hops,
and the Wilson operator of ``wilson`` becomes the 4x4 spin matrix

    D(p) = M(p) + i sum_mu gamma_mu sin p_mu,   M(p) = m + r sum_mu (1 - cos p_mu),  m = -m0,
    H(p) = gamma5 D(p),   H(p)^2 = E(p)^2 = M(p)^2 + sum_mu sin^2 p_mu,

with p_mu = 2 pi n / L_mu in the periodic directions and p_t = 2 pi (n + 1/2) / L_t
when time is antiperiodic.  Any function f of H therefore acts per momentum as

    f(H(p)) = (f(E) + f(-E))/2 + (f(E) - f(-E))/2 * H(p)/E,

which gives H_W, the exact sgn(H_W) of Eq. 2 and the quadrature operator S_N at any
lattice size without a solver (FFT over the sites).
"""
from __future__ import annotations

import numpy as np

from .gamma import gamma5, gamma_matrices

_SITE_AXES = (-6, -5, -4, -3)  # t, z, y, x in the canonical spinor layout


def _momenta(shape_tzyx, bc_t):
    lt, lz, ly, lx = shape_tzyx
    pt = 2 * np.pi * np.arange(lt) / lt
    if bc_t == -1.0:
        pt = pt + np.pi / lt
    pz = 2 * np.pi * np.arange(lz) / lz
    py = 2 * np.pi * np.arange(ly) / ly
    px = 2 * np.pi * np.arange(lx) / lx
    T, Z, Y, X = np.meshgrid(pt, pz, py, px, indexing="ij")
    return np.stack([X, Y, Z, T])  # (4 = mu, Lt, Lz, Ly, Lx)


def hamiltonian_p(shape_tzyx, m0, r=1.0, bc_t=-1.0):
    """H(p) as an array (Lt, Lz, Ly, Lx, 4, 4) and E(p) as (Lt, Lz, Ly, Lx)."""
    p = _momenta(shape_tzyx, bc_t)
    g = gamma_matrices()
    M = -m0 + r * np.sum(1.0 - np.cos(p), axis=0)
    sp = np.sin(p)
    D = M[..., None, None] * np.eye(4) + 1j * np.einsum("m...,mst->...st", sp, g)
    H = np.einsum("su,...ut->...st", gamma5(), D)
    E = np.sqrt(M**2 + np.sum(sp**2, axis=0))
    return H, E


def _twist(x, bc_t, sign):
    if bc_t != -1.0:
        return x
    lt = x.shape[-6]
    ph = np.exp(sign * 1j * np.pi * np.arange(lt) / lt)
    return x * ph.reshape((lt, 1, 1, 1, 1, 1))


def _function_p(shape_tzyx, f, m0, r, bc_t):
    """f(H(p)) as an array (Lt, Lz, Ly, Lx, 4, 4)."""
    H, E = hamiltonian_p(shape_tzyx, m0, r, bc_t)
    fp, fm = f(E), f(-E)
    return 0.5 * (fp + fm)[..., None, None] * np.eye(4) + (0.5 * (fp - fm) / E)[..., None, None] * H


def _apply_p(x, F, bc_t):
    """Apply a spin matrix per momentum, F (Lt, Lz, Ly, Lx, 4, 4), to a canonical spinor array."""
    B = np.fft.fftn(_twist(x, bc_t, -1), axes=_SITE_AXES)
    B = np.einsum("...st,...tc->...sc", F, B)
    return _twist(np.fft.ifftn(B, axes=_SITE_AXES), bc_t, +1)


def apply_function(x, f, m0, r=1.0, bc_t=-1.0):
    """f(H_W[U=1]) x for a canonical spinor array x (..., Lt, Lz, Ly, Lx, 4, 3)."""
    x = np.asarray(x, dtype=np.complex128)
    return _apply_p(x, _function_p(x.shape[-6:-2], f, m0, r, bc_t), bc_t)


def overlap_inverse(x, f, m_q, m0, r=1.0, bc_t=-1.0):
    """D_ov(m_q)^-1 x at U = 1, with the sign function replaced by f (the exact sign, or the
    rational function r_N of a quadrature): per momentum D(p) = (1 + m_q)/2 + (1 - m_q)/2
    gamma5 f(H(p)) (Eq. 1) is a 4 x 4 spin matrix, inverted directly."""
    x = np.asarray(x, dtype=np.complex128)
    S = _function_p(x.shape[-6:-2], f, m0, r, bc_t)
    D = 0.5 * (1.0 + m_q) * np.eye(4) + 0.5 * (1.0 - m_q) * np.einsum("su,...ut->...st", gamma5(), S)
    return _apply_p(x, np.linalg.inv(D), bc_t)


def apply_H(x, m0, r=1.0, bc_t=-1.0):
    """H_W[U=1] x by the momentum-space formula (f(t) = t)."""
    return apply_function(x, lambda e: e, m0, r, bc_t)


def spectrum_bounds(shape_tzyx, m0, r=1.0, bc_t=-1.0):
    """(min |lambda|, max |lambda|) of the free H_W."""
    _, E = hamiltonian_p(shape_tzyx, m0, r, bc_t)
    return float(E.min()), float(E.max())
