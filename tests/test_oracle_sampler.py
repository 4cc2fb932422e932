"""Pins of the oracle's sampler assembly: conditioning order, Markov property (brute
force Gaussian conditioning), the real DFT, and the field covariance against a direct
spherical-harmonic double sum (tiny grids, exact and sampled)."""
import math

import numpy as np
import pytest
from scipy import special

import oracle


def test_order_layout():
    k0, north, south, fn, fs = oracle.chain_layout(10, 3)
    assert k0 == 5 and north == [4, 3, 2, 1, 0] and south == [6, 7, 8, 9]
    assert [r for r, f in zip(north, fn) if f] == [2] and [r for r, f in zip(south, fs) if f] == [8]
    order = oracle.conditioning_order(10, 3)
    assert order == [5, 2, 8, 4, 3, 1, 0, 6, 7, 9]
    assert sorted(order) == list(range(10))
    # H = 0 is Alg. 2's order: equator start, then outward north, then outward south
    assert oracle.conditioning_order(7, 0) == [3, 2, 1, 0, 4, 5, 6]


def _parents(order, n_theta, H):
    """Nearest earlier neighbours of each position along z (its Markov blanket among
    the rings conditioned on before it)."""
    par = []
    for i, r in enumerate(order):
        before = order[:i]
        left = [b for b in before if b < r]
        right = [b for b in before if b > r]
        p = []
        if left:
            p.append(order.index(max(left)))
        if right:
            p.append(order.index(min(right)))
        par.append(p)
    return par


@pytest.mark.parametrize("kappa,n_theta,H,m", [([4.0], 9, 3, 2), ([3.0, 8.0], 8, 3, 1), ([3.0, 8.0], 8, 0, 3),
                                                ([2.0, 5.0, 9.0], 8, 3, 1)])
def test_markov_conditioning(kappa, n_theta, H, m):
    """Conditioning on every earlier ring equals conditioning on the nearest earlier
    neighbours on each side (the Markov property of the M-vector state, Sec. 2);
    the Cholesky diagonal blocks are the Cholesky factors of those conditional
    covariances (Eq. (innov_matrix))."""
    M = len(kappa)
    order, S, L = oracle.joint_factor(m, kappa, 1.0, n_theta, H)
    par = _parents(order, n_theta, H)
    for i in range(1, len(order)):
        allp = list(range(i))
        coef_all, cov_all = oracle.conditional_tables(S, M, i, allp)
        coef_par, cov_par = oracle.conditional_tables(S, M, i, par[i])
        # coefficients on non-parent rings vanish
        scale = np.abs(coef_all).max()
        nonpar = [j for j in allp if j not in par[i]]
        for j in nonpar:
            assert np.abs(coef_all[:, j * M:(j + 1) * M]).max() <= 1e-6 * scale
        assert np.allclose(cov_all, cov_par, rtol=1e-6, atol=1e-9 * np.abs(cov_par).max())
        Lii = L[i * M:(i + 1) * M, i * M:(i + 1) * M]
        assert np.allclose(Lii @ Lii.T, cov_all, rtol=1e-7, atol=1e-10 * np.abs(cov_all).max())


def test_dft_matches_numpy_irfft():
    rng = np.random.default_rng(0)
    N = 32
    X = rng.normal(size=N // 2 + 1) + 1j * rng.normal(size=N // 2 + 1)
    out = oracle.dft_ring(N, X.real, X.imag)
    ref = np.fft.irfft(X, n=N) * N  # irfft ignores Im X_0 and Im X_{N/2}
    assert np.allclose(out, ref, atol=1e-12)


def _ylm(l, m, theta, phi):
    """Y_lm with the paper's normalisation and Condon-Shortley phase (Sec. 2), from
    scipy's lpmv; negative m via Y_{l,-m} = (-1)^m conj(Y_lm)."""
    am = abs(m)
    n = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - am + 1) - math.lgamma(l + am + 1)))
    y = n * special.lpmv(am, l, math.cos(theta)) * np.exp(1j * am * phi)
    return y if m >= 0 else (-1) ** am * np.conj(y)


def truncated_field_cov(kappa, A, n_theta, n_phi, lmax):
    """Covariance of the discrete field by the direct double sum over (l, m) of
    C_l Y_lm(x) conj(Y_lm(y)) (Karhunen-Loeve expansion, Sec. 2), keeping |m| < n_phi/2
    and a quarter weight on m = +-n_phi/2 (the real DFT keeps Re g_{n_phi/2} (-1)^j)."""
    th = oracle.ring_theta(n_theta)
    ph = 2 * math.pi * np.arange(n_phi) / n_phi
    pts = [(t, p) for t in th for p in ph]
    Hm = n_phi // 2
    C = np.zeros((len(pts), len(pts)))
    for l in range(lmax + 1):
        cl = oracle.Cl(l, kappa, A)
        for m in range(-min(l, Hm), min(l, Hm) + 1):
            w = 0.25 if abs(m) == Hm else 1.0
            y = np.array([_ylm(l, m, t, p) for (t, p) in pts])
            C += w * cl * np.real(np.outer(y, np.conj(y)))
    return C


def exact_oracle_field_cov(kappa, A, n_theta, n_phi, H=0):
    """Field covariance implied by the oracle's factors L_m (L_m L_m^T), with its
    real-DFT synthesis written as a linear map."""
    M = len(kappa)
    Hm = n_phi // 2
    order, S, L = oracle.joint_factors(kappa, A, n_theta, n_phi, H)
    n = len(order)
    ph = 2 * math.pi * np.arange(n_phi) / n_phi
    C = np.zeros((n_theta * n_phi, n_theta * n_phi))
    for m in range(Hm + 1):
        cov = (L[m] @ L[m].T)[0::M, 0::M]  # component 0 of each position
        Cr = np.zeros((n_theta, n_theta))
        for a, ra in enumerate(order):
            for b, rb in enumerate(order):
                Cr[ra, rb] = cov[a, b]
        w = 1.0 if m == 0 else (0.5 if m == Hm else 2.0)
        ang = np.cos(m * (ph[:, None] - ph[None, :]))
        C += w * np.kron(Cr, ang)
    return C


@pytest.mark.parametrize("n_theta,n_phi,spectrum", [(3, 4, "real"), (4, 8, "real"), (4, 8, "sec5"), (4, 8, "p3")])
def test_field_covariance_tiny_bruteforce(n_theta, n_phi, spectrum):
    # C_l ~ l^-4: the direct sum converges like lmax^-3.  "sec5": the paper's Sec. 5 spectrum
    # (10 + l^2 (l+1)^2)^-1, complex kappa-hat = +-i sqrt(10); "p3": three factors, C_l ~ l^-6
    if spectrum == "real":
        kappa = [2.0, 5.0]
    elif spectrum == "p3":
        kappa = [2.0, 5.0, 9.0]
    else:
        kappa = oracle.KHat([complex(0, math.sqrt(10)), complex(0, -math.sqrt(10))])
    A = 1.0
    Cb = truncated_field_cov(kappa, A, n_theta, n_phi, 400)
    Co = exact_oracle_field_cov(kappa, A, n_theta, n_phi)
    assert np.allclose(Co, Cb, rtol=1e-6, atol=1e-6 * np.abs(Cb).max())


@pytest.mark.slow
def test_field_sample_covariance_statistical():
    """Sample covariance of 20000 oracle realisations vs the direct spherical-harmonic
    sum, within 4.5 sigma per entry (the paper's validation, Sec. 5, on a tiny grid)."""
    kappa = [2.0, 5.0]
    n_theta, n_phi, N = 4, 8, 20000
    T = oracle.sample(kappa, 1.0, n_theta, n_phi, seed=77, n_samples=N, H=0)
    X = T.reshape(N, -1)
    Cs = X.T @ X / N
    Cb = truncated_field_cov(kappa, 1.0, n_theta, n_phi, 400)
    d = np.diag(Cb)
    sig = np.sqrt((np.outer(d, d) + Cb ** 2) / N)
    z = np.abs(Cs - Cb) / sig
    assert z.max() < 4.5, z.max()
    # with the printed DFT prefactor 1/(2 m_max sqrt(2 pi)) the variance would be off by
    # a factor (2 m_max sqrt(2 pi))^2; prefactor 1 matches
    assert np.mean(np.diag(Cs)) == pytest.approx(np.mean(d), rel=0.03)


def test_anchor_order_same_law():
    """The anchored order (H > 0) and Alg. 2's order give the same field law:
    identical exact field covariances."""
    kappa = [3.0]
    C0 = exact_oracle_field_cov(kappa, 1.0, 9, 8, H=0)
    C3 = exact_oracle_field_cov(kappa, 1.0, 9, 8, H=3)
    assert np.allclose(C0, C3, rtol=1e-9, atol=1e-12 * np.abs(C0).max())


def test_im_parts_do_not_reach_field():
    # Im g_0 is identically 0 and Im g_{n_phi/2} is ignored by the real DFT
    T, X, order = oracle.sample([4.0], 1.0, 6, 8, seed=3, n_samples=2, return_coeffs=True)
    assert np.all(X[:, :, 0].imag == 0)
    c = X[0, 0].copy()
    a = oracle.dft_ring(8, c.real, c.imag)
    c2 = c.copy()
    c2[4] = c2[4].real + 123.0j
    b = oracle.dft_ring(8, c2.real, c2.imag)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n_theta,n_phi", [(3, 4), (4, 8)])
def test_field_std_is_the_mean_pointwise_variance(n_theta, n_phi):
    """field_std (the scale of every FP64 and FP32 parity tolerance) squared is the mean over
    the grid of the pointwise variance of the m-truncated field: the mean diagonal of the
    direct spherical-harmonic double sum (weights 1, 2, ..., 2, 1/2 of J^m_00 follow from the
    real-DFT convention; a wrong Nyquist weight or a lost factor 2 fails here)."""
    kappa = [2.0, 5.0]
    Cb = truncated_field_cov(kappa, 1.0, n_theta, n_phi, 400)
    v = oracle.field_std(kappa, 1.0, n_theta, n_phi) ** 2
    assert v == pytest.approx(float(np.mean(np.diag(Cb))), rel=2e-5)
    # the Nyquist term is large enough here for a wrong weight to show
    V = oracle.mode_variances(kappa, 1.0, n_theta, n_phi)
    assert 0.25 * V[-1].mean() > 1e-3 * v
