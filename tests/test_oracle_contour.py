"""Pins for the quadrature nodes, weights and rational function of Eq. 7 (CPU only)."""
import numpy as np
import pytest

from oracle import contour


@pytest.mark.parametrize("n", [4, 7, 32])
def test_circle_closed_form(n):
    """alpha = 1 (a circle): the N-point rule with the half-step offset of Eq. 7 sums
    the geometric series exactly, P_N(lambda) = 1 / (1 + ((lambda - gamma)/rho)^N)."""
    gam, rho = 0.7, 1.3
    z, p = contour.projector_coefficients(n, gam, rho, 1.0)
    lam = np.array([-2.0, -0.3, 0.1, 0.69, 1.5, 1.99, 2.5, 4.0])
    got = contour.rational(lam, z, p, 0.0)
    want = 1.0 / (1.0 + ((lam - gam) / rho) ** n)
    assert np.abs(got - want).max() < 1e-14


def test_nodes_match_eq7_parametrisation():
    z, w = contour.ellipse_nodes(8, 1.2, 1.1999, 0.1)
    th = 2 * np.pi * (np.arange(1, 9) - 0.5) / 8
    assert np.allclose(z.real, 1.2 + 1.1999 * np.cos(th))
    assert np.allclose(z.imag, 1.1999 * 0.1 * np.sin(th))
    # w_j is dz/dtheta / (i rho): the trapezoid weight of (1/2 pi i) contour integral
    dz = 1.1999 * (-np.sin(th) + 1j * 0.1 * np.cos(th))
    assert np.allclose(w, dz / (1j * 1.1999))


def test_conjugate_symmetry_makes_r_real():
    z, c, c0 = contour.single_contour(64, 3.3, 3.3, 0.28)
    assert np.allclose(z[::-1], z.conj()) and np.allclose(c[::-1], c.conj())
    lam = np.linspace(-7, 7, 301)
    assert np.abs(contour.rational(lam, z, c, c0).imag).max() < 1e-13


def test_residue_theorem_limit():
    """As N grows the rule converges to the indicator of the enclosed region."""
    z, p = contour.projector_coefficients(400, 1.2, 1.1999, 0.1)
    inside = contour.rational(np.array([0.05, 1.0, 2.3]), z, p, 0.0)
    outside = contour.rational(np.array([-0.05, -1.0, 2.5]), z, p, 0.0)
    assert np.abs(inside - 1).max() < 1e-9
    assert np.abs(outside).max() < 1e-9


def test_paper_contour_accuracy():
    """With the paper's setup (alpha = 0.1, rho = 1.1999, gamma = +-1.2) and 500 nodes
    per contour the sign function is reproduced to ~1e-14 on +-[0.01, 2]; 250 nodes
    leave ~1e-7.  This is the scalar content of the sigma-vs-N behaviour the paper reports."""
    lam = np.concatenate([np.linspace(0.01, 2.0, 400), -np.linspace(0.01, 2.0, 400)])
    z, c, c0 = contour.paper_two_contour(500)
    e500 = np.abs(contour.rational(lam, z, c, c0) - np.sign(lam)).max()
    z, c, c0 = contour.paper_two_contour(250)
    e250 = np.abs(contour.rational(lam, z, c, c0) - np.sign(lam)).max()
    assert e500 < 5e-14
    assert 1e-9 < e250 < 1e-5


def test_single_contour_is_twice_projector_minus_one():
    z, c, c0 = contour.single_contour(48, 2.0, 2.0, 0.3)
    zp, p = contour.projector_coefficients(48, 2.0, 2.0, 0.3)
    lam = np.array([-1.0, 0.5, 3.0])
    assert np.allclose(contour.rational(lam, z, c, c0), 2 * contour.rational(lam, zp, p, 0.0) - 1)


# ----------------------------------------------------------------- Zolotarev rule

def _extrema(err):
    """Values of err at its interior local extrema and the two endpoints, in order."""
    d = np.diff(err)
    idx = [0] + [k for k in range(1, len(d)) if d[k - 1] * d[k] < 0] + [len(err) - 1]
    return err[idx]


@pytest.mark.parametrize("n,b", [(3, 20.0), (4, 20.0), (5, 100.0)])
def test_zolotarev_equioscillates(n, b):
    """The optimal approximation of degree (2n-1, 2n) equioscillates: sgn - r has 2n + 1
    extrema on [1, b] with alternating signs and equal magnitude delta (Chebyshev)."""
    z, c, c0, delta = contour.zolotarev(n, 1.0, b)
    lam = np.geomspace(1.0, b, 200001)
    err = contour.rational(lam, z, c, c0).real - 1.0
    ext = _extrema(err)
    assert len(ext) == 2 * n + 1
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    assert np.allclose(np.abs(ext), delta, rtol=1e-6)
    assert np.abs(err).max() <= delta * (1 + 1e-6)


def test_zolotarev_is_odd_real_and_converges():
    deltas = []
    for n in (4, 8, 12):
        z, c, c0, delta = contour.zolotarev(n, 0.3, 6.0)
        lam = np.concatenate([np.geomspace(0.3, 6.0, 2001), -np.geomspace(0.3, 6.0, 2001)])
        r = contour.rational(lam, z, c, c0)
        assert np.abs(r.imag).max() <= 1e-13
        assert np.abs(r[:2001] + r[2001:]).max() <= 1e-13  # odd
        assert np.abs(r.real - np.sign(lam)).max() <= delta * (1 + 1e-6) + 1e-15  # + rounding of the sum
        deltas.append(delta)
    # geometric convergence in the number of poles (the rate is set by b = 20)
    assert deltas[1] < 1e-3 * deltas[0] and deltas[2] < 1e-3 * deltas[1]


def test_zolotarev_beats_trapezoid_on_spectrum():
    """On the spectrum of a small H_W (dense eigvalsh), 12 pole pairs (24 nodes) from the
    true spectral bounds approximate sgn within delta, far below a 64-node ellipse."""
    import synthetic as S
    from oracle import wilson

    U = S.su3_links((2, 2, 2, 4), 0.5, 811)
    lam = np.linalg.eigvalsh(wilson.dense_HW(U, 1.6))
    a, b = np.abs(lam).min(), np.abs(lam).max()
    z, c, c0, delta = contour.zolotarev(12, a, b)
    err = np.abs(contour.rational(lam, z, c, c0).real - np.sign(lam)).max()
    assert err <= delta * (1 + 1e-6) + 1e-15
    ze, ce, c0e = contour.single_contour(64, 0.525 * b, 0.525 * b, 0.3)
    err_e = np.abs(contour.rational(lam, ze, ce, c0e).real - np.sign(lam)).max()
    assert err < 1e-3 * err_e


# ------------------------------------- single-contour rule vs the spectral sign (Eq. 2)

def _single_contour_error(rule, n):
    """Element-wise error of the sign operator that a single-contour coefficient rule gives,
    S_N b = c0 b + sum_j c_j (z_j - H)^-1 b with one dense LU solve per node (Eqs. 5-7),
    against the spectral sign of Eq. 2, V sgn(Lambda) V^dag b (LAPACK zheevd), on a
    2x2x2x4 lattice (H_W of Eq. 1, |lambda| in [0.25, 5.9]).  The ellipse runs from 0 to
    6.8 and so encloses exactly the positive spectrum."""
    import synthetic as S
    from oracle import sign, wilson

    U = S.su3_links((2, 2, 2, 4), 0.5, 101)
    H = wilson.dense_HW(U, 1.6)
    b = S.gaussian_spinor((2, 2, 2, 4), 102).reshape(-1)
    lam, V = np.linalg.eigh(H)
    exact = V @ (np.sign(lam) * (V.conj().T @ b))
    z, c, c0 = rule(n, 3.4, 3.4, 0.3)
    s = sign.sign_apply_dense(H, b, z, c, c0)
    return np.abs(s - exact).max() / np.abs(exact).max()


def test_single_contour_pinned_to_spectral_sign():
    """sgn = 2 P_Gamma - 1 (Eq. 3 and the remark after it, P_+ + P_- = 1 without zero modes):
    the rule reaches the exact sign function of Eq. 2 within the trapezoid error, which
    falls geometrically with N (64 nodes: ~5e-7 at this gap; 192 nodes: rounding)."""
    assert _single_contour_error(contour.single_contour, 64) < 1e-5
    assert _single_contour_error(contour.single_contour, 192) < 1e-11


def _mutants():
    """Plausible slips in the single-contour rule, planted in copies of the oracle's."""
    def c0_sign(n, g, r, a):
        z, c, c0 = contour.single_contour(n, g, r, a)
        return z, c, -c0

    def no_factor_two(n, g, r, a):
        z, c, c0 = contour.single_contour(n, g, r, a)
        return z, c / 2, c0

    def conj_weights(n, g, r, a):
        z, c, c0 = contour.single_contour(n, g, r, a)
        return z, c.conj(), c0

    def neg_weights(n, g, r, a):
        z, c, c0 = contour.single_contour(n, g, r, a)
        return z, -c, c0

    def alpha_on_wrong_part_of_w(n, g, r, a):
        th = 2.0 * np.pi * (np.arange(1, n + 1) - 0.5) / n
        z = g + r * (np.cos(th) + 1j * a * np.sin(th))
        w = np.cos(th) + 1j * a * np.sin(th)
        return z, 2.0 * r * w / n, -1.0 + 0.0j

    return [c0_sign, no_factor_two, conj_weights, neg_weights, alpha_on_wrong_part_of_w]


@pytest.mark.parametrize("mutant", _mutants(), ids=lambda f: f.__name__)
def test_single_contour_pin_rejects_planted_mistakes(mutant):
    """Each planted slip moves the operator away from sgn(H) by O(1): the pin above fails it."""
    assert _single_contour_error(mutant, 64) > 1e-2
