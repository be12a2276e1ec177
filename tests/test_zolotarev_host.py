"""The library's host-side Zolotarev node generator (ov_zolotarev_rule: Jacobi elliptic
functions by the arithmetic-geometric mean, scale from the equioscillation condition)
against the oracle's (scipy elliptic functions), without a GPU."""
import numpy as np
import pytest

from oracle import contour


@pytest.fixture(scope="module")
def lib():
    from paper_2204_01583_gb300 import lib as L

    return L


@pytest.mark.parametrize("n,a,b", [(1, 1.0, 4.0), (4, 0.3, 6.0), (12, 0.3, 6.0), (16, 0.05, 6.5), (24, 0.2, 6.4)])
def test_rule_matches_oracle(lib, n, a, b):
    z, c, c0, delta = lib.zolotarev_rule(n, a, b)
    zo, co, c0o, delta_o = contour.zolotarev(n, a, b)
    assert np.abs(z - zo).max() <= 1e-12 * np.abs(zo).max()
    assert np.abs(c - co).max() <= 1e-9 * np.abs(co).max()
    # the oracle reads delta off a sampled grid, the library refines each extremum
    assert abs(delta - delta_o) <= 1e-3 * delta_o + 1e-14
    lam = np.geomspace(a, b, 20001)
    r = contour.rational(np.concatenate([lam, -lam]), z, c, c0).real
    assert np.abs(r - np.concatenate([np.ones_like(lam), -np.ones_like(lam)])).max() <= delta * (1 + 1e-6) + 1e-15


def test_rule_rejects_bad_arguments(lib):
    for args in [(0, 0.1, 1.0), (4, 0.0, 1.0), (4, 1.0, 1.0), (4, 2.0, 1.0), (129, 0.1, 1.0)]:
        with pytest.raises(lib.OvError):
            lib.zolotarev_rule(*args)
