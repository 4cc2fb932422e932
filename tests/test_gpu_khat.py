"""Spectra given by kappa-hat, including a complex-conjugate pair (Eq. (Cl); the paper's
Sec. 5 example C_l = (10 + l^2 (l+1)^2)^-1 has kappa-hat = +-i sqrt(10)) alone or beside a real
factor (p = 3): the CUDA path
through smerf_plan_create_khat against the oracle on the same seeded noise.  FP64 recursion
within 1e-10 of the field std, FP32 within 1e-4."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import oracle_field, oracle_std, rel_err

pytestmark = pytest.mark.gpu

SEC5 = (complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0)))
PAIR = (complex(40.0, 300.0), complex(40.0, -300.0))
SEC5_REAL = SEC5 + (complex(25.0, 0.0),)   # p = 3: the Sec. 5 pair and one real factor


def _plan(khat, n_theta, n_phi, H, flags=0):
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, Plan
    if H == 0:
        flags |= SMERF_ORDER_PAPER
    return Plan(A=1.0, n_theta=n_theta, n_phi=n_phi, flags=flags, anchor_spacing=H, khat=list(khat))


@pytest.mark.parametrize("khat,n_theta,n_phi,H,n,seed", [
    (SEC5, 16, 32, 0, 2, 5),      # Alg. 2's order
    (SEC5, 32, 64, 4, 3, 9),      # anchored, ragged segments
    (SEC5, 33, 64, 8, 1, 1),      # odd n_theta: start on the equator ring
    (PAIR, 24, 64, 5, 2, 3),
    (SEC5_REAL, 16, 32, 0, 2, 7),   # p = 3, Alg. 2's order
    (SEC5_REAL, 21, 64, 4, 3, 8),   # p = 3, anchored, odd n_theta
])
def test_fp64_complex_kappa_hat(khat, n_theta, n_phi, H, n, seed):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    plan = _plan(khat, n_theta, n_phi, H, SMERF_RECUR_FP64)
    got = plan.sample(seed, n).cpu().numpy()
    torch.cuda.synchronize()
    kh = oracle.KHat(khat)
    ref = oracle_field(kh, 1.0, n_theta, n_phi, seed, n, H)
    std = oracle_std(kh, 1.0, n_theta, n_phi)
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref, std) < 1e-10


def test_fp32_sec5_spectrum_64x128():
    import torch
    plan = _plan(SEC5, 64, 128, 16)
    got = plan.sample(1, 4).cpu().numpy()
    torch.cuda.synchronize()
    kh = oracle.KHat(SEC5)
    ref = oracle_field(kh, 1.0, 64, 128, 1, 4, 16)
    assert rel_err(got, ref, oracle_std(kh, 1.0, 64, 128)) < 1e-4


def test_fp32_pair_and_real_factor():
    """p = 3 with a complex-conjugate pair and a real factor, FP32 recursion, within 1e-4;
    the real factor first or last gives the same field (the set-up's partial fractions only
    change order: FP64 within 1e-10)."""
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    plan = _plan(SEC5_REAL, 24, 128, 6)
    got = plan.sample(2, 3).cpu().numpy()
    torch.cuda.synchronize()
    kh = oracle.KHat(SEC5_REAL)
    ref = oracle_field(kh, 1.0, 24, 128, 2, 3, 6)
    assert rel_err(got, ref, oracle_std(kh, 1.0, 24, 128)) < 1e-4
    a = _plan(SEC5_REAL, 16, 32, 4, SMERF_RECUR_FP64).sample(3, 2).cpu().numpy()
    b = _plan((SEC5_REAL[2],) + SEC5, 16, 32, 4, SMERF_RECUR_FP64).sample(3, 2).cpu().numpy()
    assert rel_err(a, b, float(np.std(b))) < 1e-10


def test_real_kappa_hat_is_the_kappa_plan():
    import torch
    from paper_1709_10314_gb300 import Plan
    a = Plan(A=1.0, n_theta=32, n_phi=64, anchor_spacing=8, khat=[400.0, 2500.0])
    b = Plan([20.0, 50.0], 1.0, 32, 64, anchor_spacing=8)
    assert torch.equal(a.sample(4, 3), b.sample(4, 3))


def test_rejects_other_complex_patterns():
    from paper_1709_10314_gb300 import Plan, SmerfError
    for bad in ([complex(1, 2), complex(1, 3)], [complex(1, 2), complex(2, -2)], [complex(0, 1)]):
        with pytest.raises(SmerfError):
            Plan(A=1.0, n_theta=16, n_phi=32, khat=bad)
