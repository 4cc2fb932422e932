"""The recurrence in the order m that the GPU set-up uses for real spectra (Alg. 1 sets up the
hypergeometric functions of Eq. (Legendre_hypergeometric) for every order): for
F_m(x) = 2F1(-l, l+1; 1+m; x) with l(l+1) = -kappa^2,
    F_{m-1} = [(1-2x) F_m + (1 + kappa^2/(m(m+1))) x F_{m+1}] / (1-x),
run downward from two values at the top order.  Checked here against mpmath's 2F1 (an
independent evaluation): the relation itself, the accuracy of the downward run for x < 1/2,
and its loss of accuracy for x > 1/2 (why the set-up keeps the per-mode series for a first step
whose ring lies well south of the equator)."""
import math

import pytest

mpmath = pytest.importorskip("mpmath")


def _F(kappa, m, x):
    lam = -0.5 + mpmath.sqrt(mpmath.mpf(0.25) - mpmath.mpf(kappa) ** 2)
    return mpmath.re(mpmath.hyp2f1(-lam, lam + 1, 1 + m, x))


def _down(kappa, x, mtop):
    """float64 downward run from the exact values at mtop and mtop + 1 (log-scaled as needed)."""
    Fp, F = float(_F(kappa, mtop + 1, x)), float(_F(kappa, mtop, x))
    out = {mtop + 1: Fp, mtop: F}
    for m in range(mtop, 0, -1):
        Fn = ((1 - 2 * x) * F + (1 + kappa * kappa / (m * (m + 1.0))) * x * Fp) / (1 - x)
        Fp, F = F, Fn
        out[m - 1] = F
    return out


@pytest.mark.parametrize("kappa,x,m", [(0.3, 0.2, 1), (7.0, 0.45, 3), (30.0, 0.1, 12), (80.0, 0.37, 40)])
def test_contiguous_relation(kappa, x, m):
    mpmath.mp.dps = 40
    lhs = _F(kappa, m - 1, x)
    rhs = ((1 - 2 * mpmath.mpf(x)) * _F(kappa, m, x)
           + (1 + mpmath.mpf(kappa) ** 2 / (m * (m + 1))) * x * _F(kappa, m + 1, x)) / (1 - mpmath.mpf(x))
    assert abs(lhs - rhs) <= mpmath.mpf(10) ** -30 * abs(lhs)


@pytest.mark.parametrize("kappa,x", [(20.0, 0.3), (50.0, 0.49), (5.0, 0.05)])
def test_downward_run_is_accurate_below_one_half(kappa, x):
    mpmath.mp.dps = 30
    got = _down(kappa, x, 160)
    for m in (0, 1, 7, 40, 120):
        ref = float(_F(kappa, m, x))
        assert abs(got[m] - ref) <= 1e-12 * abs(ref), (m, got[m], ref)


def test_downward_run_loses_accuracy_above_one_half():
    # errors grow by x/(1-x) per order: (0.7/0.3)^160 ~ 1e59 swamps the solution
    mpmath.mp.dps = 30
    kappa, x = 20.0, 0.7
    got = _down(kappa, x, 160)
    ref = float(_F(kappa, 0, x))
    assert not (abs(got[0] - ref) <= 1e-6 * abs(ref))
    assert 160 * math.log(x / (1 - x)) > math.log(1e3)  # the set-up's test for its first step
