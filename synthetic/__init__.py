"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module draws random numbers and builds the lattice fields that both sides
consume.  It holds none of the method's arithmetic (no Wilson operator, no
contour, no solver): only the fields the operator is applied to.

Conventions (shared by convention, not by code, with the library and the oracle):

* ``dims = (Lx, Ly, Lz, Lt)``; direction index mu = 0, 1, 2, 3 is x, y, z, t.
* Canonical gauge field: complex128 array of shape ``(4, Lt, Lz, Ly, Lx, 3, 3)``,
  ``U[mu, t, z, y, x]`` is the SU(3) matrix on the link from site x to x + mu-hat,
  row-major (row = colour index acted upon).
* Canonical spinor: complex128 array of shape ``(..., Lt, Lz, Ly, Lx, 4, 3)``,
  spin then colour, x fastest among the site indices.

The gauge links stand in for the quenched beta = 5.7 ensemble the paper uses
(Sec. "Numerical experiments"), which is not available: each link is
U = exp(i * eps * sum_a theta_a lambda_a / 2) with theta_a ~ N(0, 1), so eps sets
the roughness (eps = 0.3 ... 0.6 in the workloads), and eps = 0 is the free field.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_shape",
    "volume",
    "su3_links",
    "unit_links",
    "gaussian_spinor",
    "point_sources",
    "random_gauge_transform",
    "seed_for",
]


def lattice_shape(dims):
    """Array shape (Lt, Lz, Ly, Lx) of a lattice with dims = (Lx, Ly, Lz, Lt)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    if min(lx, ly, lz, lt) < 1:
        raise ValueError(f"bad lattice dims {dims}")
    return (lt, lz, ly, lx)


def volume(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def seed_for(tag: str, base: int = 1234) -> int:
    """Stable integer seed for a named workload (independent of PYTHONHASHSEED)."""
    h = 0
    for ch in tag.encode():
        h = (h * 131 + ch) % 1_000_003
    return base + h


def _gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _expi_hermitian(theta: np.ndarray, eps: float) -> np.ndarray:
    """exp(i * eps * sum_a theta_a lambda_a / 2) for a batch of theta[..., 8].

    Exact up to rounding: the hermitian traceless generator is diagonalised
    (LAPACK via numpy.linalg.eigh) and the phases are exponentiated.
    """
    lam = _gell_mann()
    X = np.einsum("...a,aij->...ij", theta, lam) * 0.5
    w, V = np.linalg.eigh(X)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ik,...k,...jk->...ij", V, ph, V.conj())


def su3_links(dims, eps: float, seed: int) -> np.ndarray:
    """Random SU(3) gauge field of roughness ``eps`` drawn from PCG64(seed)."""
    shp = lattice_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.standard_normal((4,) + shp + (8,))
    U = _expi_hermitian(theta, float(eps))
    return np.ascontiguousarray(U)


def unit_links(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    shp = lattice_shape(dims)
    U = np.zeros((4,) + shp + (3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_spinor(dims, seed: int, n: int | None = None) -> np.ndarray:
    """Complex Gaussian spinor(s) with E|b_i|^2 = 1, from PCG64(seed).

    Returns shape (Lt, Lz, Ly, Lx, 4, 3) if n is None, else (n, ...)."""
    shp = lattice_shape(dims) + (4, 3)
    if n is not None:
        shp = (int(n),) + shp
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    return ((re + 1j * im) / np.sqrt(2.0)).astype(np.complex128)


def point_sources(dims, site=(0, 0, 0, 0)) -> np.ndarray:
    """The 12 spin-colour point sources at one site, shape (12, Lt, Lz, Ly, Lx, 4, 3).

    Source k = 3 * spin + colour is 1 at (site, spin, colour) and 0 elsewhere;
    ``site`` is given as (x, y, z, t)."""
    shp = lattice_shape(dims)
    out = np.zeros((12,) + shp + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    for s in range(4):
        for c in range(3):
            out[3 * s + c, t, z, y, x, s, c] = 1.0
    return out


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """A random SU(3) matrix per site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    shp = lattice_shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.standard_normal(shp + (8,))
    return np.ascontiguousarray(_expi_hermitian(theta, 2.0))
