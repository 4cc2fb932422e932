"""Helpers shared by the GPU tests (the oracle side is cached per configuration)."""
import functools

import numpy as np

import oracle


@functools.lru_cache(maxsize=None)
def oracle_field(kappa, A, n_theta, n_phi, seed, n, H, rings=None):
    return oracle.sample(list(kappa), A, n_theta, n_phi, seed, n, H=H,
                         rings=None if rings is None else list(rings))


@functools.lru_cache(maxsize=None)
def oracle_std(kappa, A, n_theta, n_phi):
    return oracle.field_std(list(kappa), A, n_theta, n_phi)


def rel_err(got, ref, std):
    return float(np.max(np.abs(np.asarray(got, dtype=np.float64) - ref))) / std
