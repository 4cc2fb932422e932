"""Pin of the oracle's spectral-sum cross covariance (Lemma 2.1 in the U-basis of
Eq. (Jmatrix_more_efficient)) against the paper's closed form, Eq. (Jmatrix_efficient),
evaluated independently in multiple precision (mpmath's 2F1, Eq. (Legendre_hypergeometric))."""
import math

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")


def gauss_2f1(a, b, c, x):
    """2F1(a, b; c; x) for 0 <= x < 1: mpmath's hyp2f1, or, where it gives up (the high orders
    with arguments above about 3/4 that the large grids need), the defining Gauss series summed
    in the current precision until a term falls below 10^-(dps+5) of the sum."""
    try:
        return mp.hyp2f1(a, b, c, x)
    except mp.libmp.libhyper.NoConvergence:
        pass
    s = mp.mpc(0)
    t = mp.mpc(1)
    eps = mp.mpf(10) ** (-(mp.mp.dps + 5))
    for n in range(10 ** 6):
        s += t
        t *= (a + n) * (b + n) / ((c + n) * (n + 1)) * x
        if n > 8 and abs(t) < eps * abs(s):
            return s
    raise ArithmeticError("Gauss series did not converge")


def closed_form_J(m, kappas, A, z1, z2, p, q, dps=30, khat=None):
    """J^m_pq(z1, z2) = 1/(4 pi) sum_i b_i Gamma(1+l_i-m) Gamma(-l_i-m) *
    { (-1)^p P^{m+p}(-z1) P^{m+q}(z2)  if z1 <= z2 ;  (-1)^q P^{m+p}(z1) P^{m+q}(-z2) otherwise },
    kappa-hat_i = kappa_i^2 = -l_i (l_i + 1), b_i the partial-fraction weights (Eq. (C_ell_efficient))."""
    with mp.workdps(dps):
        tot = mp.mpf(0)
        kh = [mp.mpc(v) for v in khat] if khat is not None else [mp.mpf(k) ** 2 for k in kappas]
        for i, khi in enumerate(kh):
            b = mp.mpf(A)
            for j, khj in enumerate(kh):
                if j != i:
                    b /= khj - khi
            lam = mp.mpf(-0.5) + mp.sqrt(mp.mpf(0.25) - khi + 0j)
            G = mp.gamma(1 + lam - m) * mp.gamma(-lam - m)

            def P(mu, z):
                Q = mp.mpf(1)
                for jj in range(mu):
                    Q *= jj * (jj + 1) + khi
                return (Q / mp.factorial(mu)) * ((1 - z) / (1 + z)) ** (mp.mpf(mu) / 2) \
                    * gauss_2f1(-lam, lam + 1, 1 + mu, (1 - z) / 2)
            a1, a2 = mp.mpf(z1), mp.mpf(z2)
            if z1 <= z2:
                v = (-1) ** p * P(m + p, -a1) * P(m + q, a2)
            else:
                v = (-1) ** q * P(m + p, a1) * P(m + q, -a2)
            tot += b * G * v
        return float((tot / (4 * mp.pi)).real)


CASES = [
    ([10.0], 64, [0, 1, 7, 64]),
    ([20.0, 50.0], 32, [0, 3, 32]),
    ([3.0, 7.0], 8, [0, 2, 4]),
    ([3.0, 7.0, 15.0], 8, [0, 2, 4]),   # p = 3
]


@pytest.mark.parametrize("kappas,n_theta,ms", CASES)
def test_spectral_sum_matches_closed_form(kappas, n_theta, ms):
    th = oracle.ring_theta(n_theta)
    M = len(kappas)
    pairs = [(0, 0), (0, 1), (1, 0), (n_theta // 2, n_theta // 2 - 1), (n_theta // 2, n_theta // 2),
             (0, n_theta - 1), (2, 5)]
    S_all = oracle.cov_modes(ms, kappas, 1.0, th)
    for mi, m in enumerate(ms):
        S = S_all[mi]
        for k1, k2 in pairs:
            for p in range(M):
                for q in range(M):
                    ex = closed_form_J(m, kappas, 1.0, math.cos(th[k1]), math.cos(th[k2]), p, q)
                    got = S[k1 * M + p, k2 * M + q]
                    scale = math.sqrt(abs(S[k1 * M + p, k1 * M + p] * S[k2 * M + q, k2 * M + q]))
                    assert abs(got - ex) <= 1e-10 * scale, (m, k1, k2, p, q, got, ex)


def test_amplitude_scales_linearly():
    th = oracle.ring_theta(8)
    a = oracle.cov_m(3, [5.0], 1.0, th)
    b = oracle.cov_m(3, [5.0], 2.5, th)
    assert np.allclose(b, 2.5 * a, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_mirror_symmetry():
    # z -> -z maps the U-basis state x_q to (-1)^q x_q (the U operators are odd/even
    # under reflection), so J_pq(-z1,-z2) = (-1)^(p+q) J_pq(z1,z2) (equator symmetry, Sec. 4).
    n = 12
    th = oracle.ring_theta(n)
    M = 2
    S = oracle.cov_m(4, [4.0, 9.0], 1.0, th)
    R = oracle.cov_m(4, [4.0, 9.0], 1.0, np.pi - th)
    sgn = np.array([(-1) ** (i % M) for i in range(n * M)], dtype=float)
    assert np.allclose(R, S * np.outer(sgn, sgn), rtol=1e-10, atol=1e-12 * np.abs(S).max())


def test_windowed_sum_beats_truncation():
    # the plain partial sum of a same-point entry converges like 1/L (its tail does not
    # oscillate); the windowed + extrapolated value lies inside that tail's bracket
    th = oracle.ring_theta(64)
    z = math.cos(th[3])
    S = oracle.cov_m(2, [10.0], 1.0, th[3:4])[0, 0]
    p1 = oracle.cov_partial(2, [10.0], 1.0, z, z, 0, 0, 20000)
    p2 = oracle.cov_partial(2, [10.0], 1.0, z, z, 0, 0, 200000)
    assert p1 < p2 < S
    # 1/L tail: S - p(L) ~ c/L, so (S-p1)/(S-p2) ~ 10
    assert 8.0 < (S - p1) / (S - p2) < 12.0


KHAT_CASES = [
    # the spectrum of the paper's Sec. 5 example, C_l = (10 + l^2 (l+1)^2)^-1: kappa-hat = +-i sqrt(10)
    ([complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0))], 16, [0, 1, 5, 16]),
    ([complex(40.0, 300.0), complex(40.0, -300.0)], 32, [0, 7, 32]),
    # p = 3: the Sec. 5 pair and one real factor (kappa-hat = 25)
    ([complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0)), complex(25.0, 0.0)], 16, [0, 3, 16]),
]


@pytest.mark.parametrize("khat,n_theta,ms", KHAT_CASES)
def test_spectral_sum_matches_closed_form_complex_kappa_hat(khat, n_theta, ms):
    th = oracle.ring_theta(n_theta)
    M = len(khat)
    pairs = [(0, 0), (0, 1), (n_theta // 2, n_theta // 2 - 1), (n_theta // 2, n_theta // 2), (2, 5)]
    S_all = oracle.cov_modes(ms, oracle.KHat(khat), 1.0, th)
    for mi, m in enumerate(ms):
        S = S_all[mi]
        for k1, k2 in pairs:
            for p in range(M):
                for q in range(M):
                    ex = closed_form_J(m, None, 1.0, math.cos(th[k1]), math.cos(th[k2]), p, q, khat=khat)
                    got = S[k1 * M + p, k2 * M + q]
                    scale = math.sqrt(abs(S[k1 * M + p, k1 * M + p] * S[k2 * M + q, k2 * M + q]))
                    assert abs(got - ex) <= 1e-10 * scale, (m, k1, k2, p, q, got, ex)


def test_complex_kappa_hat_spectrum_values():
    kh = oracle.KHat([complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0))])
    for l in (0, 1, 2, 7, 100, 5000):
        L = l * (l + 1)
        assert abs(oracle.Cl(l, kh, 2.5) - 2.5 / (10.0 + L * L)) <= 1e-15 * 2.5 / (10.0 + L * L)
    # real kappa-hat given directly equals the kappa form
    for l in (0, 3, 40):
        assert oracle.Cl(l, oracle.KHat([400.0, 2500.0])) == oracle.Cl(l, [20.0, 50.0])
