"""Pins for the oracle's gamma matrices and Wilson operator (CPU only).

Each check is independent of the code it pins: Clifford algebra, hermiticity of
the dense matrix, the momentum-space free-field formula (FFT), gauge covariance
under random local SU(3) rotations, and the plain-C restatement.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import cimpl, freefield, gamma, wilson


def test_clifford_algebra():
    g = gamma.gamma_matrices()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
    g5 = gamma.gamma5()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu], -g[mu] @ g5)


def test_links_are_su3():
    U = S.su3_links((3, 2, 2, 4), 0.6, 7)
    eye = np.eye(3)
    assert np.abs(np.einsum("...ab,...cb->...ac", U, U.conj()) - eye).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    assert np.allclose(S.su3_links((2, 2, 2, 2), 0.0, 1), S.unit_links((2, 2, 2, 2)))
    assert np.array_equal(S.su3_links((2, 2, 2, 2), 0.3, 5), S.su3_links((2, 2, 2, 2), 0.3, 5))


def test_gaussian_source_variance():
    b = S.gaussian_spinor((4, 4, 4, 4), 11)
    assert abs(np.mean(np.abs(b) ** 2) - 1.0) < 0.05


@pytest.mark.parametrize("bc_t", [-1.0, 1.0])
def test_dense_HW_hermitian(bc_t):
    U = S.su3_links((2, 2, 2, 4), 0.5, 3)
    H = wilson.dense_HW(U, 1.6, bc_t=bc_t)
    assert np.abs(H - H.conj().T).max() < 1e-14


@pytest.mark.parametrize("dims,bc_t,r", [((4, 4, 2, 6), -1.0, 1.0), ((3, 4, 2, 4), 1.0, 1.0),
                                         ((4, 2, 2, 4), -1.0, 0.7)])
def test_free_field_plane_waves(dims, bc_t, r):
    psi = S.gaussian_spinor(dims, 5)
    a = wilson.apply_HW(S.unit_links(dims), psi, 1.6, r=r, bc_t=bc_t)
    b = freefield.apply_H(psi, 1.6, r=r, bc_t=bc_t)
    assert np.abs(a - b).max() < 1e-13


def test_free_field_gap():
    # p = (pi, 0, 0, p_t) branch: |m + 2 r| = 0.4 at m0 = 1.6 on a lattice with even extents
    lo, hi = freefield.spectrum_bounds((4, 4, 4, 4), 1.6, bc_t=1.0)
    assert abs(lo - 0.4) < 1e-12 and abs(hi - 6.4) < 1e-12


def test_gauge_covariance():
    dims = (2, 3, 2, 4)
    U = S.su3_links(dims, 0.6, 21)
    g = S.random_gauge_transform(dims, 22)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=-3 - mu)
        Ug[mu] = np.einsum("...ab,...bc,...dc->...ad", g, U[mu], g_fwd.conj())
    psi = S.gaussian_spinor(dims, 23)
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = wilson.apply_HW(Ug, gpsi, 1.6)
    rhs = np.einsum("...ab,...sb->...sa", g, wilson.apply_HW(U, psi, 1.6))
    assert np.abs(lhs - rhs).max() < 1e-13


@pytest.mark.parametrize("dims,bc_t", [((3, 2, 5, 4), -1), ((2, 2, 2, 2), 1), ((4, 4, 4, 4), -1)])
def test_c_oracle_matches_numpy(dims, bc_t):
    U = S.su3_links(dims, 0.5, 31)
    psi = S.gaussian_spinor(dims, 32)
    a = wilson.apply_HW(U, psi, 1.6, bc_t=float(bc_t))
    b = cimpl.hw_apply(U, psi, 1.6, bc_t=bc_t)
    assert np.abs(a - b).max() < 1e-13


def test_planted_mistake_is_caught():
    """A plausible slip (U instead of U^dag on the backward hop) breaks hermiticity."""
    dims = (2, 2, 2, 2)
    U = S.su3_links(dims, 0.5, 41)
    g = gamma.gamma_matrices()
    g5 = gamma.gamma5()

    def wrong(psi):
        out = 2.4 * psi
        for mu in range(4):
            ax = -3 - mu
            fwd = np.roll(psi, -1, axis=ax)
            bwd = np.roll(psi, +1, axis=ax)
            Ub = np.roll(U[mu], 1, axis=ax)
            hf = np.einsum("...ab,...sb->...sa", U[mu], fwd)
            hb = np.einsum("...ab,...sb->...sa", Ub, bwd)  # slip: no dagger
            out = out - 0.5 * (np.einsum("st,...tc->...sc", np.eye(4) - g[mu], hf)
                               + np.einsum("st,...tc->...sc", np.eye(4) + g[mu], hb))
        return np.einsum("st,...tc->...sc", g5, out)

    n = 12 * 16
    E = np.eye(n, dtype=np.complex128).reshape((n, 2, 2, 2, 2, 4, 3))
    Hw = wrong(E).reshape(n, n).T
    assert np.abs(Hw - Hw.conj().T).max() > 1e-3
