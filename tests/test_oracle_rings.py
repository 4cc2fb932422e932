"""Pins of the oracle's synthesis on iso-latitude grids with ring-dependent longitudes (the
paper's Sec. 1 remark: the method works on any iso-latitude grid).  Ring k keeps its latitude
theta_k and holds n_phi_ring[k] points from phi0_ring[k]; its values are the m-truncated field
evaluated there (ring_values)."""
import math

import numpy as np
import pytest
from scipy import special

import oracle


def test_full_rings_without_offset_equal_sample():
    nt, nphi = 6, 16
    full = oracle.sample([4.0], 1.0, nt, nphi, 3, 2, H=2)
    got = oracle.sample_rings([4.0], 1.0, nt, [nphi] * nt, [0.0] * nt, 3, 2, H=2)
    for j in range(2):
        for k in range(nt):
            assert np.max(np.abs(got[j][k] - full[j, k])) <= 1e-12 * np.std(full)


def test_reduced_rings_are_subsamples_and_grid_offsets_are_rolls():
    nt, nphi = 6, 16
    full = oracle.sample([3.0, 8.0], 1.0, nt, nphi, 5, 2, H=0)
    npr = [16, 8, 16, 4, 16, 8]
    sub = oracle.sample_rings([3.0, 8.0], 1.0, nt, npr, [0.0] * nt, 5, 2, H=0, n_phi=nphi)
    shift = [0, 3, 5, 1, 15, 2]
    rol = oracle.sample_rings([3.0, 8.0], 1.0, nt, [nphi] * nt, [2 * math.pi * s / nphi for s in shift], 5, 2, H=0)
    tol = 1e-12 * np.std(full)
    for j in range(2):
        for k in range(nt):
            assert np.max(np.abs(sub[j][k] - full[j, k, ::nphi // npr[k]])) <= tol
            assert np.max(np.abs(rol[j][k] - np.roll(full[j, k], -shift[k]))) <= tol


def _ylm(l, m, theta, phi):
    am = abs(m)
    n = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - am + 1) - math.lgamma(l + am + 1)))
    y = n * special.lpmv(am, l, math.cos(theta)) * np.exp(1j * am * phi)
    return y if m >= 0 else (-1) ** am * np.conj(y)


def test_offset_ring_covariance_against_spherical_harmonics():
    """Covariance of the field at half-step offsets (HEALPix-like) and on a reduced ring,
    through ring_values as a linear map of the modes' Re and Im parts and the oracle's mode
    covariances, against the direct double sum over (l, m) of C_l Y_lm Y_lm* (|m| < M) plus the
    Nyquist mode's real part, C_l Re Y_lM Re Y_lM / 2."""
    kappa, nt = [2.0, 5.0], 3
    npr, phi0 = [8, 4, 8], [math.pi / 8, math.pi / 4, 0.3]
    M = max(npr) // 2
    th = oracle.ring_theta(nt)
    pts = [(th[k], phi0[k] + 2 * math.pi * j / npr[k]) for k in range(nt) for j in range(npr[k])]
    ring_of = [k for k in range(nt) for _ in range(npr[k])]
    S = oracle.cov_modes(list(range(M + 1)), kappa, 1.0, th)  # [m][(k, q), (k', q')]
    Mq = len(kappa)
    # evaluation maps: value at each point = sum_m a_m Re g_m + b_m Im g_m (per ring)
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
        J = S[m][0::Mq, 0::Mq]  # component 0 = g_m
        Jp = J[np.ix_(ring_of, ring_of)]
        vr = 1.0 if m == 0 else 0.5      # Var(Re g_m) / J: real chain for m = 0, halves for m > 0
        vi = 0.0 if m in (0, M) else 0.5  # m = 0 and the Nyquist mode have no Im part
        C += vr * np.outer(A[:, m], A[:, m]) * Jp + vi * np.outer(B[:, m], B[:, m]) * Jp
    Cb = np.zeros_like(C)
    for l in range(401):
        cl = oracle.Cl(l, kappa)
        for m in range(-min(l, M - 1), min(l, M - 1) + 1):
            y = np.array([_ylm(l, m, t, p) for (t, p) in pts])
            Cb += cl * np.real(np.outer(y, np.conj(y)))
        if l >= M:
            yr = np.array([_ylm(l, M, t, p) for (t, p) in pts]).real
            Cb += 0.5 * cl * np.outer(yr, yr)
    assert np.allclose(C, Cb, rtol=1e-6, atol=1e-6 * np.abs(Cb).max())


def test_modes_beyond_every_ring_alias_onto_them():
    """A grid whose modes reach past every ring's own Nyquist (no ring holds n_phi points): the
    rings are still the subsamples of the full n_phi-point rings."""
    nt, nphi = 5, 32
    full = oracle.sample([6.0], 1.0, nt, nphi, 9, 1, H=0)
    npr = [4, 8, 16, 8, 4]
    sub = oracle.sample_rings([6.0], 1.0, nt, npr, [0.0] * nt, 9, 1, H=0, n_phi=nphi)
    for k in range(nt):
        assert np.max(np.abs(sub[0][k] - full[0, k, ::nphi // npr[k]])) <= 1e-12 * np.std(full)
