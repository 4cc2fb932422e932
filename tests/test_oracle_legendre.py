"""Pins for the oracle's normalised associated Legendre functions L_lm (Sec. 2):
L_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_lm, P_lm with the Condon-Shortley phase."""
import math

import numpy as np
import pytest
from scipy import special

import oracle


@pytest.mark.parametrize("m", [0, 1, 2, 5, 12])
@pytest.mark.parametrize("z", [-0.93, -0.2, 0.0, 0.41, 0.999])
def test_against_scipy_lpmv(m, z):
    lmax = 40
    row = oracle.legendre_row(m, z, lmax)
    for l in range(m, lmax + 1):
        # scipy's lpmv includes the Condon-Shortley phase, like the paper's P_lm
        ref = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1))) \
            * special.lpmv(m, l, z)
        assert row[l - m] == pytest.approx(ref, rel=1e-10, abs=1e-13)


def test_closed_forms():
    z = 0.37
    s = math.sqrt(1 - z * z)
    assert oracle.legendre_row(0, z, 1)[0] == pytest.approx(1 / math.sqrt(4 * math.pi), rel=1e-15)
    assert oracle.legendre_row(0, z, 1)[1] == pytest.approx(math.sqrt(3 / (4 * math.pi)) * z, rel=1e-15)
    assert oracle.legendre_row(1, z, 1)[0] == pytest.approx(-math.sqrt(3 / (8 * math.pi)) * s, rel=1e-15)


@pytest.mark.parametrize("m", [0, 3, 30])
def test_orthonormal_on_interval(m):
    # int_{-1}^{1} L_lm L_l'm dz = delta_ll' / (2 pi): Y_lm are orthonormal on the sphere
    x, w = np.polynomial.legendre.leggauss(200)
    lmax = m + 20
    rows = np.array([oracle.legendre_row(m, t, lmax) for t in x])
    G = (rows * w[:, None]).T @ rows
    assert np.allclose(G * 2 * math.pi, np.eye(lmax - m + 1), atol=1e-12)


def test_large_order_seed_no_underflow():
    # sin(theta)^m underflows double for m = 400 at theta = 0.01; the extended exponent
    # keeps the recurrence finite and L_lm grows back to O(1) once l sin(theta) >> m.
    m, th = 400, 0.01
    row = oracle.legendre_row(m, math.cos(th), 200000)
    assert np.all(np.isfinite(row))
    assert np.max(np.abs(row[-2000:])) > 1e-3
    # the WKB envelope at large l: mean of L^2 is about (2l+1) / (4 pi^2 sqrt(l'^2 sin^2 - m^2))
    l = np.arange(m, 200001)[-20000:]
    lp = l + 0.5
    env = (2 * l + 1) / (4 * math.pi**2 * np.sqrt(lp**2 * math.sin(th) ** 2 - m * m))
    ratio = np.mean(row[-20000:] ** 2) / np.mean(env)
    assert ratio == pytest.approx(1.0, rel=0.02)
