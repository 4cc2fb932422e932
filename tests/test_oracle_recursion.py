"""Pins of the oracle's Alg. 2 recursion (the CPU baseline of the sampler) and of its plain
FFT synthesis.  The recursion with tables from Gaussian conditioning must reproduce the dense
Cholesky factor applied to the same noise (Sec. 2: for a Markov state the factor's block rows
are exactly the transition onto the nearest earlier neighbours plus the innovation factor);
that holds only if the parents, the tables, the noise layout and the complex scaling are all
right."""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("N", [4, 8, 64, 1024])
def test_fft_ring_matches_irfft_and_dft(N):
    rng = np.random.default_rng(N)
    X = rng.normal(size=N // 2 + 1) + 1j * rng.normal(size=N // 2 + 1)
    out = oracle.fft_ring(N, X.real, X.imag)
    ref = np.fft.irfft(X, n=N) * N  # irfft ignores Im X_0 and Im X_{N/2}
    assert np.allclose(out, ref, atol=1e-11 * np.abs(ref).max())
    assert np.allclose(out, oracle.dft_ring(N, X.real, X.imag), atol=1e-11 * np.abs(ref).max())


def test_fft_ring_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft_ring(12, np.zeros(7), np.zeros(7))


CASES = [
    ([4.0], 9, 8, 0),                 # Alg. 2's order, p = 1
    ([4.0], 9, 8, 3),                 # anchored order (anchors, then bridges)
    ([3.0, 8.0], 10, 16, 0),          # p = 2
    ([3.0, 8.0], 12, 16, 4),
    ([2.0, 5.0, 9.0], 10, 16, 0),     # p = 3
    ([2.0, 5.0, 9.0], 12, 16, 4),
    (oracle.KHat([complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0))]), 8, 16, 0),  # Sec. 5
    (oracle.KHat([complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0)), 25.0]), 9, 16, 3),  # pair + real
]


@pytest.mark.parametrize("kappa,n_theta,n_phi,H", CASES)
@pytest.mark.parametrize("use_fft", [False, True])
def test_recursion_equals_dense_factor(kappa, n_theta, n_phi, H, use_fft):
    M = len(kappa)
    order, par, T, B = oracle.recursion_tables(kappa, 1.0, n_theta, n_phi, H=H)
    got = oracle.recursion_sample(M, n_phi, order, par, T, B, seed=11, n_samples=3, nthreads=2, use_fft=use_fft)
    ref = oracle.sample(kappa, 1.0, n_theta, n_phi, seed=11, n_samples=3, H=H)
    got = got[:, np.argsort(order)]  # the order's positions -> rings north to south
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.std(ref)


def test_recursion_parents_are_the_markov_blanket():
    # Alg. 2's order: every ring's parent is the previous ring of its chain, the start ring has none
    order = oracle.conditioning_order(7, 0)
    assert order == [3, 2, 1, 0, 4, 5, 6]
    assert oracle.order_parents(order) == [[], [0], [1], [2], [0], [4], [5]]
    # anchored: a bridge ring is conditioned on its inner neighbour and its outer anchor
    order = oracle.conditioning_order(10, 3)
    par = oracle.order_parents(order)
    i = order.index(4)  # between the start ring 5 and the anchor 2
    assert sorted(order[j] for j in par[i]) == [2, 5]


def test_recursion_with_a_planted_mistake_disagrees():
    """A dropped transition block (one parent's coefficients zeroed) must fail the comparison."""
    kappa, n_theta, n_phi = [4.0], 9, 8
    order, par, T, B = oracle.recursion_tables(kappa, 1.0, n_theta, n_phi, H=0)
    T = T.copy()
    T[:, 2, 0] = 0.0  # position 2 loses its parent
    got = oracle.recursion_sample(1, n_phi, order, par, T, B, seed=11, n_samples=1)[:, np.argsort(order)]
    ref = oracle.sample(kappa, 1.0, n_theta, n_phi, seed=11, n_samples=1, H=0)
    assert np.max(np.abs(got - ref)) > 1e-3 * np.std(ref)
