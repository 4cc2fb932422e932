"""Pin of the oracle's spectral sums at the orders and cut-off levels the full-size parity
tests use (Lemma 2.1 in the U-basis of Eq. (Jmatrix_more_efficient)), against the closed form
of Eq. (Jmatrix_efficient) evaluated independently in multiple precision (2F1 of
Eq. (Legendre_hypergeometric)).  At these orders the oracle's extended-exponent Legendre seeds,
its underflow cut-off and the window lengths of `default_levels` all matter; each case states
the accuracy the GPU tests rely on at that setting, in units of the diagonal scale
sqrt(J_pp(z1, z1) J_qq(z2, z2))."""
import math

import pytest

import oracle
from test_oracle_cov import closed_form_J

pytest.importorskip("mpmath")

# (kappa, n_theta, m, rings, K, level keywords, bound): the spectrum, grid and order of a
# full-size workload, the rings and levels a GPU test hands the oracle, the accuracy it needs
PINS = [
    # 1024 x 2048, p = 2: start ring (default levels), a first band, sampled bridge tables (K = 4)
    ([20.0, 50.0], 1024, 1024, [512], 6, {}, 1e-10),
    ([20.0, 50.0], 1024, 700, [512, 511, 510], 6, {}, 1e-10),
    ([20.0, 50.0], 1024, 517, [495, 496, 480], 4, {}, 1e-9),
    ([20.0, 50.0], 1024, 1024, [497, 498, 496], 4, {}, 1e-9),
    # 4096 x 8192, p = 1: start ring of the precision sweep (K = 4, c_turn_diag = 16)
    ([100.0], 4096, 512, [2048], 4, dict(c_turn_diag=16.0), 2e-8),
    ([100.0], 4096, 4096, [2048], 4, dict(c_turn_diag=16.0), 2e-8),
    # 16384 x 32768, p = 1: start ring (K = 5, c_turn_diag = 8), ring variances (K = 4,
    # c_turn_diag = 4) on and away from the equator, sampled bridge tables (default levels)
    ([300.0], 16384, 4096, [8192], 5, dict(c_turn_diag=8.0), 2e-8),
    ([300.0], 16384, 16384, [8192], 5, dict(c_turn_diag=8.0), 2e-8),
    ([300.0], 16384, 0, [4000], 4, dict(c_turn_diag=4.0), 2e-5),
    ([300.0], 16384, 16384, [8192], 4, dict(c_turn_diag=4.0), 2e-5),
    ([300.0], 16384, 16384, [4000], 4, dict(c_turn_diag=4.0), 2e-5),
    ([300.0], 16384, 4000, [8183, 8184, 8176], 6, {}, 1e-10),
    ([300.0], 16384, 16384, [8171, 8172, 8160], 6, {}, 1e-10),
    # stepped-ring parity grids (tests/test_gpu_stepped.py): 48 x 2048, p = 2, anchors every 16
    # rings (start ring, both anchors, the first bridge rings; K = 4, c_turn_diag = 8), and
    # 4 x 32768, p = 1 (start ring and its neighbour; K = 4, c_turn_diag = 4)
    ([20.0, 50.0], 48, 300, [24, 8, 40, 23, 22], 4, dict(c_turn_diag=8.0), 1e-6),
    ([20.0, 50.0], 48, 1024, [24, 8, 40, 23, 22], 4, dict(c_turn_diag=8.0), 1e-6),
    ([300.0], 4, 4000, [2, 1], 4, dict(c_turn_diag=4.0), 2e-5),
    ([300.0], 4, 16384, [2, 1], 4, dict(c_turn_diag=4.0), 2e-5),
    # 24 x 16384, p = 1, anchors every 8 rings: start ring, anchors, first bridge rings
    ([300.0], 24, 3000, [12, 4, 20, 11, 10], 4, dict(c_turn_diag=4.0), 2e-5),
    ([300.0], 24, 8192, [12, 4, 20, 11, 10], 4, dict(c_turn_diag=4.0), 2e-5),
    # p = 3 parity grids (tests/test_gpu_p3.py): 6 x 4096 with anchors every 2 rings (start
    # ring, an anchor, a bridge ring) and 4 x 8192 in Alg. 2's order (K = 4, c_turn_diag = 8)
    ([4.0, 9.0, 20.0], 6, 700, [3, 1, 2], 4, dict(c_turn_diag=8.0), 3e-6),
    ([4.0, 9.0, 20.0], 6, 2048, [3, 1, 2], 4, dict(c_turn_diag=8.0), 3e-6),
    ([4.0, 9.0, 20.0], 4, 1500, [2, 1], 4, dict(c_turn_diag=8.0), 3e-6),
    ([4.0, 9.0, 20.0], 4, 4096, [2, 1], 4, dict(c_turn_diag=8.0), 3e-6),
]


@pytest.mark.parametrize("kappa,n_theta,m,rings,K,kw,bound", PINS)
def test_high_order_spectral_sums(kappa, n_theta, m, rings, K, kw, bound):
    th = oracle.ring_theta(n_theta)[rings]
    M = len(kappa)
    S = oracle.cov_modes([m], kappa, 1.0, th, K=K, **kw)[0]
    worst = 0.0
    for a in range(len(rings)):
        for b in range(len(rings)):
            for p in range(M):
                for q in range(M):
                    ex = closed_form_J(m, kappa, 1.0, math.cos(th[a]), math.cos(th[b]), p, q)
                    scale = math.sqrt(abs(S[a * M + p, a * M + p] * S[b * M + q, b * M + q]))
                    worst = max(worst, abs(S[a * M + p, b * M + q] - ex) / scale)
    assert worst <= bound, (kappa, n_theta, m, rings, K, kw, worst)


def test_reduced_levels_are_not_enough():
    """The pin has teeth: the cut-offs that are too short for this grid (K = 3,
    c_turn_diag = 2) miss the closed form at m = 16384 by far more than any bound above."""
    th = oracle.ring_theta(16384)[[8192]]
    S = oracle.cov_modes([16384], [300.0], 1.0, th, K=3, c_turn_diag=2.0)[0]
    ex = closed_form_J(16384, [300.0], 1.0, math.cos(th[0]), math.cos(th[0]), 0, 0)
    assert abs(S[0, 0] - ex) / S[0, 0] > 1e-3
