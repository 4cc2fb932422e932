"""Pins for the oracle's noise: Philox4x32-10 and Box-Muller (not in the paper, which
only asks for standard normal samples, Eq. (state_space) and Alg. 2)."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key) == expect


def test_ring_counter_and_key_layout():
    # call j of ring k under 64-bit key K uses counter (j, k, 0, 0), key (K lo, K hi)
    K = 0x0123456789ABCDEF
    raw = oracle.raw_uint32(K, 7, 3)
    for j in range(3):
        assert list(raw[4 * j:4 * j + 4]) == oracle.philox4x32_10([j, 7, 0, 0], [K & 0xFFFFFFFF, K >> 32])


def test_normals_distribution():
    from scipy import stats
    x = np.concatenate([oracle.ring_normals(1234 + s, k, 4096) for s in range(4) for k in range(16)])
    assert x.size == 4 * 16 * 4096
    assert abs(x.mean()) < 5.0 / math.sqrt(x.size)
    assert abs(x.var() - 1.0) < 6.0 * math.sqrt(2.0 / x.size)
    ks = stats.kstest(x, "norm")
    assert ks.pvalue > 1e-3
    # pairs from one Philox call are uncorrelated
    y = x.reshape(-1, 4)
    c = np.corrcoef(y.T)
    assert np.max(np.abs(c - np.eye(4))) < 5.0 / math.sqrt(y.shape[0])


def test_rings_and_keys_independent():
    a = oracle.ring_normals(1, 0, 1000)
    b = oracle.ring_normals(1, 1, 1000)
    c = oracle.ring_normals(2, 0, 1000)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15
