"""Quadrature of the contour-integral projector (oracle; test infrastructure only).

Eq. 7: with theta_j = 2 pi (j - 1/2) / N_q, j = 1..N_q,

    z_j = gamma + rho (cos theta_j + i alpha sin theta_j)      (nodes on an ellipse)
    w_j = alpha cos theta_j + i sin theta_j
    P_Gamma x  ~=  (1 / N_q) sum_j rho w_j y_j,   (z_j - H) y_j = x   (Eq. 6)

A sign-function coefficient list (z_j, c_j, c0) represents the operator
S_N = c0 * 1 + sum_j c_j (z_j - H)^-1, whose value on an eigenvalue lambda is the
scalar rational function r_N(lambda) = c0 + sum_j c_j / (z_j - lambda).

* ``paper_two_contour``: Eq. 3 and Eq. 5, sgn = P_+ - P_-, one ellipse around the
  positive and one around the negative spectrum (centres +gamma and -gamma); c0 = 0.
* ``single_contour``: sgn = 2 P_+ - 1, valid when H has no exact zero mode
  (P_+ + P_- = 1 minus the kernel projector, Eq. 3 and the remark after it); c0 = -1.
"""
from __future__ import annotations

import numpy as np


def ellipse_nodes(n_q: int, gamma: float, rho: float, alpha: float):
    """(z_j, w_j), j = 1..n_q, of Eq. 7."""
    j = np.arange(1, n_q + 1, dtype=np.float64)
    theta = 2.0 * np.pi * (j - 0.5) / n_q
    z = gamma + rho * (np.cos(theta) + 1j * alpha * np.sin(theta))
    w = alpha * np.cos(theta) + 1j * np.sin(theta)
    return z.astype(np.complex128), w.astype(np.complex128)


def projector_coefficients(n_q: int, gamma: float, rho: float, alpha: float):
    """(z_j, rho w_j / N_q): the quadrature of P_Gamma in Eq. 7."""
    z, w = ellipse_nodes(n_q, gamma, rho, alpha)
    return z, rho * w / n_q


def single_contour(n_q: int, gamma: float, rho: float, alpha: float):
    """sgn = 2 P_Gamma - 1 with Gamma around the positive spectrum: (z, c, c0)."""
    z, p = projector_coefficients(n_q, gamma, rho, alpha)
    return z, 2.0 * p, -1.0 + 0.0j


def paper_two_contour(n_q: int, gamma: float = 1.2, rho: float = 1.1999, alpha: float = 0.1):
    """sgn = P_{Gamma+} - P_{Gamma-} (Eqs. 3, 5): n_q nodes on each ellipse.

    Defaults are the paper's integration setup (Supplement, "Numerical setup
    for the integration"): alpha = 0.1, rho = 1.1999, centres +-1.2."""
    zp, pp = projector_coefficients(n_q, +gamma, rho, alpha)
    zm, pm = projector_coefficients(n_q, -gamma, rho, alpha)
    return np.concatenate([zp, zm]), np.concatenate([pp, -pm]), 0.0 + 0.0j


def rational(lam, z, c, c0):
    """r_N(lambda) = c0 + sum_j c_j / (z_j - lambda), the value of S_N on an eigenvalue."""
    lam = np.asarray(lam, dtype=np.complex128)
    return c0 + np.sum(c[None, :] / (z[None, :] - lam.reshape(-1, 1)), axis=1).reshape(lam.shape)


def zolotarev(n_poles: int, lam_min: float, lam_max: float, samples: int = 400001):
    """Zolotarev's optimal uniform rational approximation of sgn(lambda) on
    [-lam_max, -lam_min] u [lam_min, lam_max], written as a resolvent sum (z, c, c0 = 0).

    Not in the paper (which names better contour rules as future work in its
    "Summary"); this is the classical construction.  With x = lambda / lam_min,
    b = lam_max / lam_min, parameter m' = 1 - 1/b^2, K' = K(m'), and
    c_l = sn^2(l K' / 2n | m') / cn^2(l K' / 2n | m'), l = 1 .. 2n - 1,

        R(x) = d0 x prod_{i=1}^{n-1} (x^2 + c_{2i}) / prod_{i=1}^{n} (x^2 + c_{2i-1})
             = x sum_{l=1}^{n} b_l / (x^2 + c_{2l-1}),

    with d0 set so that R - 1 equioscillates between -delta and +delta on [1, b] (found
    here by dense sampling in log x).  Since lam / (lam^2 + s^2) =
    -1/2 [1 / (i s - lam) + 1 / (-i s - lam)], each pole pair gives the nodes
    z = +-i s_l, s_l = lam_min sqrt(c_{2l-1}), both with coefficient -b_l lam_min / 2.
    Returns (z, c, c0, delta), nodes ordered i s_1 .. i s_n, -i s_n .. -i s_1."""
    from scipy.special import ellipj, ellipk

    n = int(n_poles)
    b = lam_max / lam_min
    m1 = 1.0 - 1.0 / b**2
    K1 = ellipk(m1)
    sn, cn, _, _ = ellipj(np.arange(1, 2 * n) * K1 / (2 * n), m1)
    cl = sn**2 / cn**2
    codd, ceven = cl[0::2], cl[1::2]
    x = np.geomspace(1.0, b, samples)
    Rt = x * np.prod(x[:, None] ** 2 + ceven[None, :], axis=1) / np.prod(x[:, None] ** 2 + codd[None, :], axis=1)
    lo, hi = Rt.min(), Rt.max()
    d0 = 2.0 / (lo + hi)
    delta = (hi - lo) / (hi + lo)
    bl = np.array([d0 * np.prod(ceven - co) / np.prod(np.delete(codd, i) - co) for i, co in enumerate(codd)])
    s = lam_min * np.sqrt(codd)
    z = np.concatenate([1j * s, -1j * s[::-1]])
    c = np.concatenate([-0.5 * lam_min * bl, -0.5 * lam_min * bl[::-1]]).astype(np.complex128)
    return z.astype(np.complex128), c, 0.0 + 0.0j, float(delta)
