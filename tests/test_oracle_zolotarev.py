"""Pins of the oracle's Zolotarev coefficients: by the alternation theorem the
best uniform approximation of type (2n+1, 2n) has an error curve with 2n+2
alternating extrema of equal size. A wrong pole, residue or scale breaks the
equal ripple; the partial fractions must equal the product form."""
import numpy as np
import pytest

from oracle import zolotarev


def _alternation(co, k, grid=400001):
    lam = np.exp(np.linspace(0.0, np.log(1.0 / k), grid))
    e = 1.0 - zolotarev.rational_sign_product(lam, co, 1.0)
    s = np.sign(np.diff(e))
    idx = np.where(s[1:] != s[:-1])[0] + 1
    return np.concatenate([[e[0]], e[idx], [e[-1]]])


@pytest.mark.parametrize("k,n", [(0.05, 3), (0.01, 4), (0.2, 2), (0.1, 5), (0.02, 6)])
def test_equioscillation(k, n):
    co = zolotarev.zolotarev_coefficients(k, n)
    ext = _alternation(co, k)
    assert len(ext) == 2 * n + 2
    assert np.all(np.sign(ext[1:]) == -np.sign(ext[:-1]))
    assert np.allclose(np.abs(ext), co["delta"], rtol=1e-5)


def test_partial_fractions_equal_product():
    co = zolotarev.zolotarev_coefficients(0.03, 12)
    lam = np.exp(np.linspace(np.log(0.5), np.log(1 / 0.03 * 1.5), 1001))
    a = zolotarev.rational_sign_scalar(lam, co, 1.0)
    b = zolotarev.rational_sign_product(lam, co, 1.0)
    assert np.allclose(a, b, rtol=1e-12)


def test_error_falls_with_degree_and_odd_symmetry():
    d = [zolotarev.zolotarev_coefficients(0.05, n)["delta"] for n in (2, 4, 8)]
    assert d[0] > d[1] > d[2]
    co = zolotarev.zolotarev_coefficients(0.05, 6)
    lam = np.linspace(1, 20, 50)
    assert np.allclose(zolotarev.rational_sign_scalar(-lam, co, 1.0),
                       -zolotarev.rational_sign_scalar(lam, co, 1.0))
    assert np.all(co["c_den"] > 0) and np.all(np.diff(co["c_den"]) > 0)
