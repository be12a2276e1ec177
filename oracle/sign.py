"""Sign function and overlap operator from resolvents (oracle; test infrastructure only).

Steps, in the paper's order:

1. nodes and weights of the contour (Eq. 7, ``contour``);
2. for every node, the resolvent solve (z_j I - H_W) y_j = x (Eq. 6), here each
   node solved on its own: dense LU (numpy.linalg.solve) on tiny lattices, CGNR
   on the normal equations otherwise;
3. the weighted sum sgn(H_W) x ~= c0 x + sum_j c_j y_j (Eqs. 5, 7);
4. D_ov(m_q) x = (1 + m_q)/2 x + (1 - m_q)/2 gamma5 sgn(H_W) x (Eq. 1).

Also the exact spectral sign function of Eq. 2, the quality measure sigma and the
Ginsparg-Wilson residual of Sec. "Numerical experiments".
"""
from __future__ import annotations

import numpy as np

from . import contour
from .gamma import gamma5
from .wilson import apply_HW


# ---------------------------------------------------------------- dense forms

def resolvents_dense(H, x, z):
    """y_j = (z_j I - H)^-1 x for every node (Eq. 6), one LU solve per node."""
    n = H.shape[0]
    eye = np.eye(n, dtype=np.complex128)
    return np.stack([np.linalg.solve(zj * eye - H, x) for zj in z])


def sign_apply_dense(H, x, z, c, c0):
    """S_N x = c0 x + sum_j c_j (z_j - H)^-1 x (Eqs. 5, 7) with dense per-node solves."""
    y = resolvents_dense(H, x, z)
    return c0 * x + np.tensordot(c, y, axes=(0, 0))


def spectral_function(H, f):
    """V f(Lambda) V^dag from the dense eigendecomposition H = V Lambda V^dag (LAPACK zheevd)."""
    lam, V = np.linalg.eigh(H)
    return (V * f(lam)[None, :]) @ V.conj().T, lam


def spectral_sign(H):
    """sgn(H) = sum_i sgn(lambda_i) v_i v_i^dag (Eq. 2), with sgn(0) = 0."""
    S, _ = spectral_function(H, np.sign)
    return S


# ------------------------------------------------------ iterative (any size)

def cgnr_solve(U, x, zj, m0, r=1.0, bc_t=-1.0, tol=1e-13, maxiter=100000):
    """Solve (zj - H_W) y = x by CG on the normal equations (CGNR / CGLS).

    A = zj - H_W is normal with A^dag = conj(zj) - H_W.  Iterates minimise
    ||x - A y|| over growing Krylov spaces of A^dag A; stops when the recursive
    residual ||x - A y|| <= tol ||x||, then returns (y, iterations, true relative residual).
    """
    def A(v):
        return zj * v - apply_HW(U, v, m0, r, bc_t)

    def AH(v):
        return np.conj(zj) * v - apply_HW(U, v, m0, r, bc_t)

    bn = np.linalg.norm(x)
    y = np.zeros_like(x)
    res = x.copy()
    s = AH(res)
    p = s.copy()
    gam = np.vdot(s, s).real
    it = 0
    while np.linalg.norm(res) > tol * bn and it < maxiter:
        q = A(p)
        a = gam / np.vdot(q, q).real
        y = y + a * p
        res = res - a * q
        s = AH(res)
        gnew = np.vdot(s, s).real
        p = s + (gnew / gam) * p
        gam = gnew
        it += 1
    true_res = np.linalg.norm(x - A(y)) / bn
    return y, it, true_res


def sign_apply(U, x, z, c, c0, m0, r=1.0, bc_t=-1.0, tol=1e-13):
    """S_N x on a canonical spinor array, one CGNR solve per node (Eqs. 5-7)."""
    out = c0 * np.asarray(x, dtype=np.complex128)
    for zj, cj in zip(z, c):
        y, _, _ = cgnr_solve(U, x, zj, m0, r, bc_t, tol)
        out = out + cj * y
    return out


# ------------------------------------------------------------ overlap and checks

def g5(x):
    """gamma5 on the spin axis of a canonical spinor array (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", gamma5(), x)


def overlap_from_sign(x, s, m_q):
    """D_ov(m_q) x = (1 + m_q)/2 x + (1 - m_q)/2 gamma5 s with s = sgn(H_W) x (Eq. 1)."""
    return 0.5 * (1.0 + m_q) * x + 0.5 * (1.0 - m_q) * g5(s)


def sigma(y, s):
    """Quality of the sign function: |s^dag s - y^dag y| / y^dag y with s = sgn(H) y."""
    yy = np.vdot(y, y).real
    return abs(np.vdot(s, s).real - yy) / yy


def overlap_dense(H, z, c, c0, m_q):
    """Dense D_ov(m_q) = (1 + m_q)/2 + (1 - m_q)/2 gamma5 S_N (Eq. 1), with the quadrature
    operator S_N = V r_N(Lambda) V^dag, r_N(lambda) = c0 + sum_j c_j / (z_j - lambda)
    (Eqs. 5, 7 on the eigenbasis of H).  Tiny lattices only."""
    lam, V = np.linalg.eigh(H)
    rN = contour.rational(lam, z, c, c0)
    S = (V * rN[None, :]) @ V.conj().T
    n = H.shape[0]
    g = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), n // 12)
    return 0.5 * (1.0 + m_q) * np.eye(n) + 0.5 * (1.0 - m_q) * g[:, None] * S


def overlap_solve_dense(H, b, z, c, c0, m_q):
    """x = D_ov(m_q)^-1 b by LU on the dense operator: the solve the overlap propagator
    needs (each of its matrix-vector products is one D_ov apply, Eq. 1)."""
    return np.linalg.solve(overlap_dense(H, z, c, c0, m_q), np.asarray(b, dtype=np.complex128).reshape(-1))


def gw_residual(apply_D0, x):
    """(gamma5 D + D gamma5 - 2 D gamma5 D) x for the massless overlap operator D.

    The paper prints the Ginsparg-Wilson relation without the factor 2; with the
    1/2 normalisation of Eq. 1 the relation that holds is {D, gamma5} = 2 D gamma5 D."""
    Dx = apply_D0(x)
    return g5(Dx) + apply_D0(g5(x)) - 2.0 * apply_D0(g5(Dx))
