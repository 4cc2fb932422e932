"""Oracle on HEALPix grids (the iso-latitude grids of the paper's Sec. 1 remark): rings at the
HEALPix colatitudes with 4i points in the polar caps and 4 Nside in the equatorial belt, each
offset by half a pixel where HEALPix offsets it.  Pinned against the direct spherical-harmonic
double sum of the field covariance at the pixel centres (Nside = 3: rings of 4, 8 and 12 points)
and, with the equiangular colatitudes given explicitly, against the default grid."""
import math

import numpy as np
import pytest
from scipy import special

import oracle


def healpix_rings(nside):
    """Colatitudes, point counts and first-pixel longitudes of the 4 nside - 1 HEALPix rings,
    north to south (Gorski et al. 2005: polar ring i < nside at z = 1 - i^2 / (3 nside^2) with 4i
    pixels at phi = pi (j - 1/2) / (2i); equatorial ring nside <= i <= 2 nside at
    z = 4/3 - 2i / (3 nside) with 4 nside pixels at phi = pi (j - s/2) / (2 nside),
    s = (i - nside + 1) mod 2; the southern rings mirror the northern ones)."""
    z, n, p0 = [], [], []
    for i in range(1, 2 * nside + 1):
        if i < nside:
            z.append(1.0 - i * i / (3.0 * nside * nside))
            n.append(4 * i)
            p0.append(math.pi / (4.0 * i))
        else:
            z.append(4.0 / 3.0 - 2.0 * i / (3.0 * nside))
            n.append(4 * nside)
            s = (i - nside + 1) % 2
            p0.append(math.pi * s / (4.0 * nside))
    # mirror the northern rings (all but the equator ring i = 2 nside) to the south
    zs = z + [-v for v in reversed(z[:-1])]
    ns = n + list(reversed(n[:-1]))
    ps = p0 + list(reversed(p0[:-1]))
    return np.arccos(np.array(zs)), ns, ps


def _ylm(l, m, theta, phi):
    am = abs(m)
    n = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - am + 1) - math.lgamma(l + am + 1)))
    y = n * special.lpmv(am, l, math.cos(theta)) * np.exp(1j * am * phi)
    return y if m >= 0 else (-1) ** am * np.conj(y)


def test_healpix_ring_layout():
    th, n, p0 = healpix_rings(3)
    assert len(th) == 11 and sum(n) == 12 * 9
    assert np.allclose(th + th[::-1], math.pi)   # symmetric about the equator
    assert np.all(np.diff(th) > 0)


@pytest.mark.parametrize("n_rings", [11, 7])
def test_healpix_covariance_against_spherical_harmonics(n_rings):
    """The covariance of the oracle's field at the HEALPix pixel centres (Nside = 3, modes up to
    the grid's n_phi / 2 = 6, the rings of 4 and 8 points aliasing the modes above their own
    Nyquist) against the direct double sum over (l, m) of C_l Y_lm Y_lm* (|m| < 6) plus the
    Nyquist mode's real part; on all 11 rings, and on the 7 northern ones (a grid that is not
    symmetric about the equator)."""
    kappa = [2.0, 5.0]
    th, npr, phi0 = healpix_rings(3)
    th, npr, phi0 = th[:n_rings], npr[:n_rings], phi0[:n_rings]
    nt, nphi = len(th), 12
    M = nphi // 2
    pts = [(th[k], phi0[k] + 2 * math.pi * j / npr[k]) for k in range(nt) for j in range(npr[k])]
    ring_of = [k for k in range(nt) for _ in range(npr[k])]
    S = oracle.cov_modes(list(range(M + 1)), kappa, 1.0, th)
    Mq = len(kappa)
    A = np.zeros((len(pts), M + 1))
    B = np.zeros((len(pts), M + 1))
    row = 0
    for k in range(nt):
        for m in range(M + 1):
            e = np.zeros(M + 1, dtype=complex)
            e[m] = 1.0
            A[row:row + npr[k], m] = oracle.ring_values(e, npr[k], phi0[k])
            e[m] = 1j
            B[row:row + npr[k], m] = oracle.ring_values(e, npr[k], phi0[k])
        row += npr[k]
    C = np.zeros((len(pts), len(pts)))
    for m in range(M + 1):
        Jp = S[m][0::Mq, 0::Mq][np.ix_(ring_of, ring_of)]
        vr = 1.0 if m == 0 else 0.5
        vi = 0.0 if m in (0, M) else 0.5
        C += vr * np.outer(A[:, m], A[:, m]) * Jp + vi * np.outer(B[:, m], B[:, m]) * Jp
    Cb = np.zeros_like(C)
    for l in range(401):
        cl = oracle.Cl(l, kappa)
        ys = {m: np.array([_ylm(l, m, t, p) for (t, p) in pts]) for m in range(0, min(l, M) + 1)}
        for m in range(-min(l, M - 1), min(l, M - 1) + 1):
            y = ys[abs(m)] if m >= 0 else (-1) ** abs(m) * np.conj(ys[abs(m)])
            Cb += cl * np.real(np.outer(y, np.conj(y)))
        if l >= M:
            yr = ys[M].real
            Cb += 0.5 * cl * np.outer(yr, yr)
    assert np.allclose(C, Cb, rtol=1e-6, atol=1e-6 * np.abs(Cb).max())


def test_equiangular_theta_given_explicitly_is_the_default_grid():
    th = oracle.ring_theta(9)
    a = oracle.sample([4.0], 1.0, 9, 16, 5, 2, H=3)
    b = oracle.sample([4.0], 1.0, 9, 16, 5, 2, H=3, theta=list(th))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("H", [0, 3])
def test_healpix_samples_are_the_factor_on_the_noise(H):
    """sample_rings on the HEALPix rings (custom colatitudes, 12-point rings) equals Alg. 2's
    recursion with tables from the same colatitudes, synthesised at the same points."""
    th, npr, phi0 = healpix_rings(3)
    nt = len(th)
    got = oracle.sample_rings([3.0, 7.0], 1.0, nt, npr, phi0, 4, 2, H=H, n_phi=16, theta=th)
    _, X, order = oracle.sample([3.0, 7.0], 1.0, nt, 16, 4, 2, H=H, return_coeffs=True, theta=th)
    pos = {r: i for i, r in enumerate(order)}
    for j in range(2):
        for k in range(nt):
            ref = oracle.ring_values(X[j, pos[k]], npr[k], phi0[k])
            assert np.allclose(got[j][k], ref, rtol=0, atol=1e-14)


def test_start_ring():
    """Alg. 2 starts at the equator: n_theta // 2 on a symmetric grid, else the ring nearest it
    (the southern one of two at the same distance)."""
    assert oracle.start_ring(9) == 4 and oracle.start_ring(10) == 5
    th, _, _ = healpix_rings(3)
    assert oracle.start_ring(11, th) == 5
    assert oracle.start_ring(4, [0.2, 0.5, 0.9, 1.3]) == 3            # a northern band: its last ring
    assert oracle.start_ring(3, [2.0, 2.5, 3.0]) == 0                 # a southern band: its first ring
    assert oracle.start_ring(4, [0.3, 1.5, 1.7, 2.0]) == 1            # straddling, nearer the north
    h = math.pi / 2
    assert oracle.start_ring(4, [0.3, h - 0.1, h + 0.1, 2.0]) == 2    # a tie: the southern ring
    k0, north, south, _, _ = oracle.chain_layout(4, 0, [0.2, 0.5, 0.9, 1.3])
    assert (k0, north, south) == (3, [2, 1, 0], [])


BANDS = [
    ([4.0], [0.25, 0.4, 0.6, 0.75, 0.95, 1.1, 1.3], 8, 0),              # northern band: one chain
    ([3.0, 8.0], [0.25, 0.4, 0.6, 0.75, 0.95, 1.1, 1.3], 16, 3),
    ([2.0, 5.0, 9.0], [0.5, 0.8, 1.2, 1.5, 1.75, 2.1, 2.3, 2.6], 16, 3),  # straddling, uneven steps
    ([3.0, 8.0], [1.9, 2.1, 2.2, 2.5, 2.8], 16, 0),                     # southern band
]


@pytest.mark.parametrize("kappa,theta,n_phi,H", BANDS)
def test_band_recursion_equals_dense_factor(kappa, theta, n_phi, H):
    """On grids that are not symmetric about the equator the recursion from the start ring
    nearest the equator, with tables from Gaussian conditioning, reproduces the dense factor on
    the same noise: the order keeps the Markov property (Sec. 2) wherever the chains start."""
    nt = len(theta)
    order, par, T, B = oracle.recursion_tables(kappa, 1.0, nt, n_phi, H=H, theta=theta)
    assert order[0] == oracle.start_ring(nt, theta)
    got = oracle.recursion_sample(len(kappa), n_phi, order, par, T, B, seed=5, n_samples=2, use_fft=True)
    ref = oracle.sample(kappa, 1.0, nt, n_phi, seed=5, n_samples=2, H=H, theta=theta)
    got = got[:, np.argsort(order)]
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.std(ref)
