"""GPU set-up tables (FP64) against the oracle's brute-force Gaussian conditioning of the
spectral-sum joint covariance (Eqs. (trans_matrix), (innov_matrix), (state_initial)).

Compared in standardised units: regression coefficients scaled by the parent's and the
child's standard deviations, conditional covariances by the child's."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _ring_pos(order):
    return {r: i for i, r in enumerate(order)}


def _check_block(S, M, pos, parents, A_gpu, C_gpu, B_gpu, sign, tol, m):
    coef, cov = oracle.conditional_tables(S, M, pos, parents)
    sd = lambda i: np.sqrt(np.diag(S)[i * M:(i + 1) * M])
    sc = sd(pos)
    Sg = np.diag(sign)
    half = 0.5 if m > 0 else 1.0
    # the southern chain's tables act on S x: A = S A_gpu S etc.
    blocks = [A_gpu] + ([C_gpu] if C_gpu is not None else [])
    for b, par in enumerate(parents):
        got = Sg @ blocks[b] @ Sg
        ref = coef[:, b * M:(b + 1) * M]
        sp = sd(par)
        err = np.abs(got - ref) * sp[None, :] / sc[:, None]
        assert err.max() < tol, ("coef", m, pos, b, err.max())
    Bg = Sg @ B_gpu  # stored southern factors carry S in their columns
    covg = Bg @ Bg.T / half
    err = np.abs(covg - cov) / np.outer(sc, sc)
    assert err.max() < tol, ("cov", m, pos, err.max())


def _unpack(rowvals, M, kind):
    """rows of one mode -> (A, C, B) for steps, (A, B) for coarse, B for the start."""
    tri = [(p, q) for p in range(M) for q in range(p + 1)]
    def lower(v):
        L = np.zeros((M, M))
        for (p, q), x in zip(tri, v):
            L[p, q] = x
        return L
    if kind == "step":
        return rowvals[:M * M].reshape(M, M), rowvals[M * M:2 * M * M].reshape(M, M), lower(rowvals[2 * M * M:])
    if kind == "coarse":
        return rowvals[:M * M].reshape(M, M), lower(rowvals[M * M:])
    return lower(rowvals)


@pytest.mark.parametrize("kappa,n_theta,H", [([6.0], 12, 0), ([6.0], 12, 4), ([3.0, 8.0], 12, 4),
                                             ([3.0, 8.0], 13, 3), ([20.0, 50.0], 16, 0)])
def test_tables_match_gaussian_conditioning(kappa, n_theta, H):
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_ORDER_PAPER, Plan
    M = len(kappa)
    n_phi = 16
    flags = SMERF_RECUR_FP64 | (SMERF_ORDER_PAPER if H == 0 else 0)
    plan = Plan(kappa, 1.0, n_theta, n_phi, flags=flags, anchor_spacing=H if H else 0)
    info = plan.info()
    order, Ss, _ = oracle.joint_factors(kappa, 1.0, n_theta, n_phi, H=H)
    pos_of = _ring_pos(order)
    k0, north, south, fn, fs = oracle.chain_layout(n_theta, H)
    beq = plan.tables(0)
    tol = 2e-8
    for m in range(n_phi // 2 + 1):
        S = Ss[m]
        half = 0.5 if m > 0 else 1.0
        B0 = _unpack(beq[:, m], M, "start")
        cov0 = S[:M, :M]
        assert np.abs(B0 @ B0.T / half - cov0).max() / np.abs(cov0).max() < tol
        for c, (ch, fl) in enumerate([(north, fn), (south, fs)]):
            sign = np.array([(-1) ** q if c == 1 else 1 for q in range(M)], dtype=float)
            anchors = [i + 1 for i, f in enumerate(fl) if f]   # positions
            assert info["n_anchors"][c] == len(anchors)
            for p in range(1, len(ch) + 1):
                if p in anchors:
                    continue
                ring = ch[p - 1]
                left = k0 if p == 1 else ch[p - 2]
                right = [a for a in anchors if a > p]
                A_, C_, B_ = _unpack(plan.tables(1, c, p)[:, m], M, "step")
                if right:
                    par = [pos_of[left], pos_of[ch[right[0] - 1]]]
                    _check_block(S, M, pos_of[ring], par, A_, C_, B_, sign, tol, m)
                else:
                    assert np.abs(C_).max() <= 2.0 ** -119  # zeros are stored as 2^-120
                    _check_block(S, M, pos_of[ring], [pos_of[left]], A_, None, B_, sign, tol, m)
            for j, a in enumerate(anchors):
                A_, B_ = _unpack(plan.tables(2, c, j + 1)[:, m], M, "coarse")
                prev = k0 if j == 0 else ch[anchors[j - 1] - 1]
                _check_block(S, M, pos_of[ch[a - 1]], [pos_of[prev]], A_, None, B_, sign, tol, m)


@pytest.mark.parametrize("kappa", [[40.0], [150.0], [20.0, 50.0], [40.0, 130.0]])
def test_tables_at_high_orders(kappa):
    # step tables (real spectra) come from a downward recurrence over every order m (Alg. 1
    # with the contiguous relation); check them at orders spread over 0..512 on a 24-ring grid
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_ORDER_PAPER, Plan
    M, n_theta, n_phi = len(kappa), 24, 1024
    plan = Plan(kappa, 1.0, n_theta, n_phi, flags=SMERF_RECUR_FP64 | SMERF_ORDER_PAPER, anchor_spacing=0)
    ms = [0, 1, 2, 37, 200, 511, 512]
    order, Ss, _ = oracle.joint_factors(kappa, 1.0, n_theta, n_phi, H=0, modes=ms)
    pos_of = _ring_pos(order)
    k0, north, south, _, _ = oracle.chain_layout(n_theta, 0)
    for i, m in enumerate(ms):
        S = Ss[i]
        for c, ch in enumerate([north, south]):
            sign = np.array([(-1.0) ** q if c == 1 else 1.0 for q in range(M)])
            for p in range(1, len(ch) + 1):
                left = k0 if p == 1 else ch[p - 2]
                A_, C_, B_ = _unpack(plan.tables(1, c, p)[:, m], M, "step")
                _check_block(S, M, pos_of[ch[p - 1]], [pos_of[left]], A_, None, B_, sign, 2e-8, m)
