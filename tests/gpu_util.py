"""Helpers shared by the GPU tests (the oracle side is cached per configuration)."""
import functools

import numpy as np

import oracle


def _k(kappa):
    """The oracle's spectrum argument: a KHat as it is, real kappa as a list."""
    return kappa if isinstance(kappa, oracle.KHat) else list(kappa)


@functools.lru_cache(maxsize=None)
def oracle_field(kappa, A, n_theta, n_phi, seed, n, H, rings=None):
    return oracle.sample(_k(kappa), A, n_theta, n_phi, seed, n, H=H,
                         rings=None if rings is None else list(rings))


@functools.lru_cache(maxsize=None)
def oracle_std(kappa, A, n_theta, n_phi):
    return oracle.field_std(_k(kappa), A, n_theta, n_phi)


def rel_err(got, ref, std):
    return float(np.max(np.abs(np.asarray(got, dtype=np.float64) - ref))) / std
