"""Oracle for the sphere-GMRF sampler (arXiv 1709.10314).  TEST INFRASTRUCTURE ONLY.

What it computes, step by step, in the paper's notation:

1. Spectrum C_l = A / prod_i (l(l+1) + kappa-hat_i)            -- Eq. (Cl); kappa-hat_i = kappa_i^2
   for a list of real kappa, or complex kappa-hat given as KHat([...]) (real values or
   complex-conjugate pairs, so that C_l is real; Sec. 5 uses +-i sqrt(10)).
2. For each azimuthal mode m = 0..n_phi/2, the joint covariance of the U-basis state
   vector g_m^{(0..M-1)} at every ring, by direct spectral summation over normalised
   associated Legendre functions                              -- Lemma 2.1 + Eq. (Jmatrix_more_efficient)
   (C core: oracle_cov_m; windowed sum + Richardson in 1/L on same-ring blocks).
3. The states are ordered in the sampler's conditioning order (the start ring, the
   anchor rings of the northern and southern chains, then every other ring outward);
   dense Cholesky of that matrix is sequential Gaussian conditioning in that order
   (Eqs. (trans_matrix), (innov_matrix), (state_initial)), which for a Markov state
   reproduces the recursion's map from white noise to states  -- Eq. (state_space).
4. The factor is applied to the same Philox4x32-10 / Box-Muller noise the sampler
   draws (Re and Im chains of a mode m > 0 take half the covariance: complex standard
   normal noise, Sec. 2 after Eq. (state_space)).
5. Each ring is synthesised by a naive real DFT with prefactor 1 -- Alg. 2, last step.

Pins (tests/test_oracle_*.py, run with -m "not gpu"):
  philox4x32_10            pinned: published known-answer vectors (Random123 / SC'11)
  ring_normals             pinned: KS test against the normal CDF, moment checks
  legendre_row             pinned: scipy.special.lpmv, closed forms for small l
  cov_m                    pinned: closed-form Green's function (Eq. (Jmatrix_efficient))
                           evaluated independently with mpmath, at grid points (one, two and
                           three spectrum factors; orders up to 16384 at the GPU tests' levels)
  sample / chol            pinned: brute-force Gaussian conditioning (Markov property),
                           sample covariance vs the m-truncated analytic covariance,
                           tiny-grid brute force over (l, m) spherical-harmonic sums,
                           Im(g_0) and Im(g_{n_phi/2}) invariants
  start_ring               pinned: the equator ring (or the first south of it) on symmetric
                           grids, the ring nearest the equator on bands; the recursion from it
                           equals the dense factor on northern, southern and straddling bands
  dft_ring                 pinned: numpy.fft.irfft (library routine)
  fft_ring                 pinned: numpy.fft.irfft and dft_ring
  recursion_sample         pinned: equals sample() (the dense factor applied to the same
                           noise) on small grids in both orders and for p = 1, 2, 3, which
                           holds only if the tables, the parents and the noise layout are all right
  ring_values /            pinned: full rings without offset equal sample(); a ring of n_phi/2
  sample_rings             points is every second point of the full ring; an offset of s grid
                           steps is the full ring rolled by s; the field covariance at offset
                           points equals the direct spherical-harmonic double sum (tiny grids)
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "philox4x32_10", "raw_uint32", "ring_normals", "Cl", "legendre_row",
    "cov_partial", "cov_m", "default_levels", "ring_theta", "start_ring", "chain_layout",
    "conditioning_order", "normal_index", "joint_factor", "joint_factors", "cov_modes",
    "sample", "field_std", "mode_variances",
    "conditional_tables", "dft_ring", "fft_ring", "KHat",
    "order_parents", "recursion_tables", "recursion_sample",
    "ring_values", "sample_rings",
]

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_ring_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, dp]
        L.oracle_raw_uint32.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, u32p]
        L.oracle_Cl.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double]
        L.oracle_Cl.restype = ctypes.c_double
        L.oracle_cov_m.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
                                   dp, ctypes.c_long, lp, ctypes.c_int, dp]
        L.oracle_cov_m.restype = ctypes.c_int
        L.oracle_cov_modes.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, dp,
                                       ctypes.c_double, ctypes.c_int, dp, lp, lp, ctypes.c_int, dp]
        L.oracle_cov_modes.restype = ctypes.c_int
        L.oracle_cov_partial.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_long]
        L.oracle_cov_partial.restype = ctypes.c_double
        L.oracle_legendre_row.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]
        L.oracle_dft_ring.argtypes = [ctypes.c_int, dp, dp, dp]
        L.oracle_fft_ring.argtypes = [ctypes.c_int, dp, dp, dp]
        L.oracle_fft_ring.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_recursion_sample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip, ip, dp, dp,
                                              ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.oracle_recursion_sample.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------ noise
def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter under a 2-word key (Salmon et al., SC'11)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def raw_uint32(key64, ring, ncalls):
    out = np.zeros(4 * ncalls, dtype=np.uint32)
    lib().oracle_raw_uint32(ctypes.c_uint64(key64 & (2**64 - 1)), ring, ncalls,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def ring_normals(key64, ring, n):
    """First n standard normals of ring `ring` for Philox key `key64`.
    Call j uses counter (j, ring, 0, 0); Box-Muller maps its words (0,1) and (2,3)
    to normals 4j, 4j+1 and 4j+2, 4j+3."""
    out = np.zeros(n, dtype=np.float64)
    lib().oracle_ring_normals(ctypes.c_uint64(key64 & (2**64 - 1)), ring, n, _dp(out))
    return out


def normal_index(n_phi, M, m, part, q):
    """Index, within a ring's normals, of the normal driving component q of the
    Re (part=0) or Im (part=1) chain of mode m.  Slot s = m for 1 <= m < n_phi/2
    takes normals [2Ms, 2Ms+2M): Re first, then Im.  Slot 0 holds the real chain of
    m = 0 (normals [0, M)) and the Re chain of the Nyquist mode m = n_phi/2
    (normals [M, 2M)); their Im chains do not reach the field."""
    H = n_phi // 2
    if m == 0:
        assert part == 0
        return q
    if m == H:
        assert part == 0
        return M + q
    return 2 * M * m + M * part + q


# --------------------------------------------------------------- spectrum
class KHat(tuple):
    """kappa-hat_i given directly (complex allowed), in place of a list of real kappa."""


def _spec(kappa):
    """The C core's spectrum argument: kappa-hat_i as (re, im) pairs, and p."""
    if isinstance(kappa, KHat):
        kh = [complex(v) for v in kappa]
    else:
        kh = [complex(float(k) * float(k), 0.0) for k in np.atleast_1d(np.asarray(kappa, dtype=np.float64))]
    out = np.zeros(2 * len(kh))
    out[0::2] = [v.real for v in kh]
    out[1::2] = [v.imag for v in kh]
    return np.ascontiguousarray(out), len(kh)


def Cl(l, kappa, A=1.0):
    k, M = _spec(kappa)
    return lib().oracle_Cl(int(l), M, _dp(k), float(A))


def legendre_row(mu, z, lmax):
    """Normalised L_{l,mu}(z), l = mu..lmax, Condon-Shortley phase (Sec. 2)."""
    out = np.zeros(lmax - mu + 1)
    lib().oracle_legendre_row(mu, float(z), lmax, _dp(out))
    return out


def cov_partial(m, kappa, A, z1, z2, p, q, lmax):
    """Plain partial sum of J^m_pq(z1, z2) up to l = lmax (no window)."""
    k, M = _spec(kappa)
    return lib().oracle_cov_partial(m, M, _dp(k), float(A), float(z1), float(z2), p, q, int(lmax))


def default_levels(m, M, theta, c_turn_off=8.0, c_turn_diag=32.0, c_osc=400.0, lmin=2000):
    """Cut-offs for the windowed sums at ring angles theta.

    Off-diagonal blocks only oscillate in l (frequencies |t1-t2|, t1+t2, 2pi-t1-t2);
    a smooth window suppresses their tail once L*frequency >> 1 and L/2 is well past
    every turning point l ~ m/sin(theta).  Same-ring blocks carry a non-oscillating
    1/l^2 tail that the Richardson extrapolation in 1/L removes; they need L well past
    the turning point of that ring."""
    th = np.asarray(theta, dtype=np.float64)
    s = np.sin(th)
    mm = m + M
    tt = np.unique(th)
    if tt.size > 1:
        dmin = float(np.min(np.diff(np.sort(tt))))
    else:
        dmin = math.pi
    wmin = min(dmin, 2 * float(tt.min()), 2 * (math.pi - float(tt.max())))
    Loff = int(max(lmin, c_turn_off * mm / float(s.min()), c_osc / wmin))
    wdiag = np.minimum(2 * th, 2 * (math.pi - th))
    Ld = np.maximum(np.maximum(lmin, c_turn_diag * mm / s), c_osc / wdiag).astype(np.int64)
    return Loff, Ld


def cov_m(m, kappa, A, theta, K=6, levels=None):
    """Joint covariance of the U-basis state of mode m at rings theta (any order).
    Returns (n*M, n*M), index (k*M+p, k2*M+q)."""
    k, M = _spec(kappa)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    z = np.ascontiguousarray(np.cos(th))
    n = len(z)
    Loff, Ld = levels if levels is not None else default_levels(m, M, th)
    Ld = np.ascontiguousarray(Ld, dtype=np.int64)
    S = np.zeros((n * M, n * M))
    rc = lib().oracle_cov_m(m, M, _dp(k), float(A), n, _dp(z), int(Loff),
                            Ld.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), int(K), _dp(S))
    if rc != 0:
        raise ValueError("oracle_cov_m: bad arguments")
    return S


def cov_modes(ms, kappa, A, theta, K=6, **level_kw):
    """cov_m for every mode in `ms` (computed in parallel in the C core).
    Returns an array [len(ms), n*M, n*M]."""
    k, M = _spec(kappa)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    z = np.ascontiguousarray(np.cos(th))
    n = len(z)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    Loff = np.zeros(len(ms), dtype=np.int64)
    Ld = np.zeros((len(ms), n), dtype=np.int64)
    for i, m in enumerate(ms):
        Loff[i], Ld[i] = default_levels(int(m), M, th, **level_kw)
    out = np.zeros((len(ms), n * M, n * M))
    rc = lib().oracle_cov_modes(len(ms), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), M, _dp(k),
                                float(A), n, _dp(z), Loff.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                Ld.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), int(K), _dp(out))
    if rc != 0:
        raise ValueError("oracle_cov_modes: bad arguments")
    return out


# ------------------------------------------------------------ grid, order
def ring_theta(n_theta, theta=None):
    """Cell-centred equiangular rings theta_k = pi (k + 1/2) / n_theta, k = 0..n_theta-1
    (north to south).  The paper's grid (Sec. 4) is garbled in print; this is the
    symmetric reading with no pole rings.  `theta` (n_theta colatitudes, increasing in
    (0, pi)) replaces them on other iso-latitude grids (Sec. 1 remark: the method needs
    only rings of constant latitude), e.g. HEALPix, or a band of latitudes."""
    if theta is None:
        return math.pi * (np.arange(n_theta) + 0.5) / n_theta
    th = np.asarray(theta, dtype=np.float64)
    assert th.shape == (n_theta,)
    return th


def start_ring(n_theta, theta=None):
    """Alg. 2 builds outward from the equator.  On a grid symmetric about it (the default
    grid; given colatitudes with theta_k + theta_{n_theta-1-k} = pi within 1e-12 pi) the
    start ring is n_theta // 2: the equator ring for odd n_theta, the first ring south of
    it for even n_theta.  On any other grid it is the ring nearest the equator, the
    southern one of two at the same distance."""
    if theta is None:
        return n_theta // 2
    th = np.asarray(theta, dtype=np.float64)
    if all(abs(th[k] + th[n_theta - 1 - k] - math.pi) <= 1e-12 * math.pi for k in range(n_theta)):
        return n_theta // 2
    d = [abs(t - math.pi / 2) for t in th]
    return max(k for k in range(n_theta) if d[k] == min(d))


def chain_layout(n_theta, H, theta=None):
    """Start ring k0 (start_ring) and the two chains: the northern chain visits
    k0-1, ..., 0 and the southern chain k0+1, ..., n_theta-1 (Alg. 2 builds outward
    from the equator).  Anchors sit every H rings along each chain (H <= 0 or
    H >= n_theta: none, which is exactly Alg. 2's order).
    Returns (k0, [north rings], [south rings], [north anchor flags], [south anchor flags])."""
    k0 = start_ring(n_theta, theta)
    north = [k0 - i for i in range(1, k0 + 1)]
    south = [k0 + i for i in range(1, n_theta - k0)]
    use = 0 < H < n_theta

    def flags(ch):
        return [use and ((i + 1) % H == 0) for i in range(len(ch))]
    return k0, north, south, flags(north), flags(south)


def conditioning_order(n_theta, H, theta=None):
    """Rings in the order the sampler conditions on them: the start ring, the northern
    anchors outward, the southern anchors outward, then every other northern ring
    outward, then every other southern ring outward.  Each ring's conditional law given
    all earlier rings equals its law given its nearest earlier neighbours (Markov
    property of the state, Sec. 2), which is what the sampler uses."""
    k0, north, south, fn, fs = chain_layout(n_theta, H, theta)
    order = [k0]
    order += [r for r, f in zip(north, fn) if f]
    order += [r for r, f in zip(south, fs) if f]
    order += [r for r, f in zip(north, fn) if not f]
    order += [r for r, f in zip(south, fs) if not f]
    return order


# --------------------------------------------------------------- factor
def joint_factors(kappa, A, n_theta, n_phi, H=0, K=6, rings=None, modes=None, theta=None, **level_kw):
    """Dense lower Cholesky factors of every mode's joint state covariance in
    conditioning order (Cholesky = sequential Gaussian conditioning,
    Eqs. (trans_matrix), (innov_matrix), (state_initial)).  `rings` restricts to a
    leading subset of that order, whose factor is the leading block of the full one.
    Returns (order, [Sigma_m], [L_m]) for m in `modes` (default 0..n_phi/2)."""
    order = conditioning_order(n_theta, H, theta) if rings is None else list(rings)
    th = ring_theta(n_theta, theta)[order]
    ms = list(range(n_phi // 2 + 1)) if modes is None else list(modes)
    S = cov_modes(ms, kappa, A, th, K=K, **level_kw)
    Ls = [np.linalg.cholesky(S[i]) for i in range(len(ms))]
    return order, [S[i] for i in range(len(ms))], Ls


def joint_factor(m, kappa, A, n_theta, H=0, K=6, rings=None, **level_kw):
    order, S, L = joint_factors(kappa, A, n_theta, 2, H, K, rings, modes=[m], **level_kw)
    return order, S[0], L[0]


def conditional_tables(S, M, pos, parents):
    """Gaussian conditioning of the state at position `pos` on the states at
    positions `parents` (Eqs. (trans_matrix), (innov_matrix)): returns (coef, cov)
    with E[x_pos | x_par] = coef @ x_par and Cov = cov."""
    ix = np.arange(pos * M, pos * M + M)
    jx = np.concatenate([np.arange(p * M, p * M + M) for p in parents]) if len(parents) else np.zeros(0, int)
    Skk = S[np.ix_(ix, ix)]
    if len(jx) == 0:
        return np.zeros((M, 0)), Skk
    Skj = S[np.ix_(ix, jx)]
    Sjj = S[np.ix_(jx, jx)]
    coef = np.linalg.solve(Sjj, Skj.T).T
    cov = Skk - coef @ Skj.T
    return coef, cov


def fft_ring(N, re, im):
    """The real synthesis of dft_ring through a plain radix-2 FFT (N a power of two)."""
    re = np.ascontiguousarray(re, dtype=np.float64)
    im = np.ascontiguousarray(im, dtype=np.float64)
    out = np.zeros(N)
    if lib().oracle_fft_ring(N, _dp(re), _dp(im), _dp(out)) != 0:
        raise ValueError("oracle_fft_ring: N must be a power of two")
    return out


def dft_ring(N, re, im):
    re = np.ascontiguousarray(re, dtype=np.float64)
    im = np.ascontiguousarray(im, dtype=np.float64)
    out = np.zeros(N)
    lib().oracle_dft_ring(N, _dp(re), _dp(im), _dp(out))
    return out


# --------------------------------------------------------------- sample
def sample(kappa, A, n_theta, n_phi, seed, n_samples=1, H=0, K=6, rings=None,
           factors=None, return_coeffs=False, theta=None, **level_kw):
    """Realisations j = 0..n_samples-1 with Philox key seed + j.

    Returns float64 [n_samples][n_rings][n_phi]: every ring north to south (default),
    or the rings of `rings` (a leading subset of the conditioning order) in that order."""
    M = _spec(kappa)[1]
    Hm = n_phi // 2
    order_full = conditioning_order(n_theta, H, theta)
    if rings is None:
        order = order_full
    else:
        order = list(rings)
        assert order == order_full[:len(order)], "rings must be a leading subset of the order"
    if factors is None:
        factors = joint_factors(kappa, A, n_theta, n_phi, H, K, rings=order, theta=theta, **level_kw)[2]
    n = len(order)
    out_rings = sorted(order) if rings is None else order
    pos = {r: i for i, r in enumerate(order)}
    need = M * n_phi
    half = 1.0 / math.sqrt(2.0)
    # noise: [realisation][position in order][normal index within the ring]
    nrm = np.zeros((n_samples, n, need))
    for j in range(n_samples):
        key = (seed + j) & (2**64 - 1)
        for i, r in enumerate(order):
            nrm[j, i] = ring_normals(key, r, need)
    X = np.zeros((n_samples, n, Hm + 1), dtype=np.complex128)
    for m in range(Hm + 1):
        Lf = factors[m]

        def chain(part):
            cols = [normal_index(n_phi, M, m, part, q) for q in range(M)]
            xi = nrm[:, :, cols].reshape(n_samples, n * M)   # state order (position, component)
            return (xi @ Lf.T).reshape(n_samples, n, M)[:, :, 0]
        if m == 0:
            X[:, :, m] = chain(0)
        elif m == Hm:
            X[:, :, m] = chain(0) * half
        else:
            X[:, :, m] = (chain(0) + 1j * chain(1)) * half
    res = np.zeros((n_samples, len(out_rings), n_phi))
    for j in range(n_samples):
        for oi, r in enumerate(out_rings):
            c = X[j, pos[r]]
            res[j, oi] = dft_ring(n_phi, c.real, c.imag)
    if return_coeffs:
        return res, X, order
    return res


def mode_variances(kappa, A, n_theta, n_phi, K=6, rings=None, theta=None, **level_kw):
    """J^m_00(z_k, z_k) = E|g_m(z_k)|^2 for m = 0..n_phi/2 at the given rings
    (Lemma 2.1).  Returns [n_phi/2+1][n_rings]."""
    M = _spec(kappa)[1]
    idx = list(range(n_theta)) if rings is None else list(rings)
    th = ring_theta(n_theta, theta)[idx]
    ms = list(range(n_phi // 2 + 1))
    out = np.zeros((len(ms), len(idx)))
    for i, t in enumerate(th):
        S = cov_modes(ms, kappa, A, np.array([t]), K=K, **level_kw)
        out[:, i] = S[:, 0, 0]
    return out


def field_std(kappa, A, n_theta, n_phi, K=6, rings=None, theta=None):
    """Root of the ring-mean pointwise variance of the discrete field:
    mean_k [J^0_00 + 2 sum_{0<m<n_phi/2} J^m_00 + J^{n_phi/2}_00 / 2], the variance of
    the m-truncated field with the real-DFT convention (Lemma 2.1)."""
    V = mode_variances(kappa, A, n_theta, n_phi, K, rings, theta=theta)
    Hm = n_phi // 2
    w = np.full(Hm + 1, 2.0)
    w[0] = 1.0
    w[Hm] = 0.5
    return float(math.sqrt((w[:, None] * V).sum(axis=0).mean()))


# ------------------------------------------------------- Alg. 2 with tables
def order_parents(order):
    """For each position of a conditioning order, its nearest earlier neighbours in ring
    index on each side (at most two): the Markov blanket among the rings drawn before it
    (Sec. 2), i.e. the parents of the recursion x_i = sum_j T_ij x_par(j) + B_i xi_i."""
    par = []
    for i, r in enumerate(order):
        before = order[:i]
        lo = [b for b in before if b < r]
        hi = [b for b in before if b > r]
        p = []
        if hi:
            p.append(order.index(min(hi)))
        if lo:
            p.append(order.index(max(lo)))
        par.append(p)
    return par


def recursion_tables(kappa, A, n_theta, n_phi, H=0, K=6, rings=None, modes=None, theta=None, **level_kw):
    """Tables of Alg. 2's recursion for every mode and every position of the conditioning
    order (or of its leading subset `rings`), from the oracle's joint covariance: the
    transition onto each parent by Gaussian conditioning (Eq. (trans_matrix)) and, as the
    innovation factor (Eq. (innov_matrix)), the position's diagonal block of the dense
    lower Cholesky factor (the factor of the conditional covariance).
    Returns (order, parents, T [n_modes][n_pos][2][M][M], B [n_modes][n_pos][M][M]) for the
    modes `modes` (default 0..n_phi/2)."""
    M = _spec(kappa)[1]
    order, S, L = joint_factors(kappa, A, n_theta, n_phi, H, K, rings=rings, modes=modes, theta=theta, **level_kw)
    par = order_parents(order)
    n = len(order)
    T = np.zeros((len(S), n, 2, M, M))
    B = np.zeros((len(S), n, M, M))
    for mi in range(len(S)):
        for i in range(n):
            B[mi, i] = L[mi][i * M:(i + 1) * M, i * M:(i + 1) * M]
            if par[i]:
                coef, _ = conditional_tables(S[mi], M, i, par[i])
                for j in range(len(par[i])):
                    T[mi, i, j] = coef[:, j * M:(j + 1) * M]
    return order, par, T, B


def recursion_sample(M, n_phi, order, parents, T, B, seed, n_samples=1, nthreads=1, use_fft=True):
    """Alg. 2: the per-sample recursion over the positions of `order` with the given tables
    (recursion_tables), the same Philox noise as sample(), and the per-ring synthesis
    (fft_ring, or the naive dft_ring).  Returns float64 [n_samples][len(order)][n_phi], rings
    in the order's order."""
    n = len(order)
    ring = np.ascontiguousarray(order, dtype=np.int32)
    npar = np.ascontiguousarray([len(p) for p in parents], dtype=np.int32)
    par = np.zeros((n, 2), dtype=np.int32)
    for i, p in enumerate(parents):
        par[i, :len(p)] = p
    T = np.ascontiguousarray(T, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert T.shape[0] == n_phi // 2 + 1 and T.shape[1] == n and B.shape[:2] == T.shape[:2]
    out = np.zeros((n_samples, n, n_phi))
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().oracle_recursion_sample(M, n_phi, n, ring.ctypes.data_as(ip), npar.ctypes.data_as(ip),
                                       par.ctypes.data_as(ip), _dp(T), _dp(B),
                                       ctypes.c_uint64(seed & (2**64 - 1)), n_samples, int(nthreads),
                                       1 if use_fft else 0, _dp(out))
    if rc != 0:
        raise ValueError("oracle_recursion_sample: bad arguments")
    return out


# ------------------------------------------------ iso-latitude grids (Sec. 1 remark)
def ring_values(c, n, phi0):
    """The m-truncated field on one ring at the n points phi_j = phi0 + 2 pi j / n, from its
    coefficients c[m] = g_m, m = 0..M (M = len(c) - 1): the real field
        T(phi) = g_0 + 2 sum_{0<m<M} Re(g_m e^{i m phi}) + Re(g_M) cos(M phi),
    the full ring's convention (prefactor 1, Alg. 2; the Nyquist coefficient's real part) at any
    phi.  Evaluated directly, O(M n); modes above the ring's own Nyquist alias as the sum says."""
    c = np.asarray(c, dtype=np.complex128)
    M = len(c) - 1
    phi = phi0 + 2.0 * math.pi * np.arange(n) / n
    m = np.arange(1, M)
    E = np.exp(1j * np.outer(phi, m))
    out = np.full(n, c[0].real)
    out += 2.0 * (E @ c[1:M]).real
    out += c[M].real * np.cos(M * phi)
    return out


def sample_rings(kappa, A, n_theta, n_phi_ring, phi0_ring, seed, n_samples=1, H=0, K=6, rings=None,
                 n_phi=None, theta=None, **level_kw):
    """Realisations on an iso-latitude grid with ring-dependent longitudes: ring k (colatitude
    theta_k = pi (k + 1/2) / n_theta, or theta[k]) holds n_phi_ring[k] points starting at
    phi0_ring[k] (any even count: ring_values evaluates the field at each point).  The
    modes m = 0..n_phi/2 (n_phi defaults to max(n_phi_ring)), their recursion and noise are those
    of sample() on the n_theta x n_phi grid; each ring is synthesised at its own points
    (ring_values).  Returns a list over realisations of lists of ring arrays, rings north to south
    (or in the order of `rings`, a leading subset of the conditioning order)."""
    n_phi = int(max(n_phi_ring)) if n_phi is None else int(n_phi)
    assert max(n_phi_ring) <= n_phi
    _, X, order = sample(kappa, A, n_theta, n_phi, seed, n_samples, H=H, K=K, rings=rings,
                         return_coeffs=True, theta=theta, **level_kw)
    out_rings = sorted(order) if rings is None else list(rings)
    pos = {r: i for i, r in enumerate(order)}
    res = []
    for j in range(n_samples):
        res.append([ring_values(X[j, pos[r]], int(n_phi_ring[r]), float(phi0_ring[r])) for r in out_rings])
    return res
