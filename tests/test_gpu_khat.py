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


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("khat,grid,n_phi,H", [
    (SEC5, "healpix3", 16, 3),      # the Sec. 5 spectrum at the Nside 3 HEALPix colatitudes
    (PAIR, "band", 64, 0),          # a pair on a band that straddles the equator unevenly
    (SEC5_REAL, "band", 32, 4),     # p = 3: the pair and a real factor
])
def test_complex_kappa_hat_at_given_colatitudes(fp64, khat, grid, n_phi, H):
    """smerf_plan_create_khat_theta: complex kappa-hat on the rings of another iso-latitude grid
    (the set-up's complex construction at the given colatitudes) against the oracle."""
    import torch
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, SMERF_RECUR_FP64, Plan
    if grid == "healpix3":
        from test_oracle_healpix import healpix_rings
        theta = list(healpix_rings(3)[0])
    else:
        theta = [0.35, 0.6, 0.8, 1.05, 1.3, 1.62, 1.8, 2.05, 2.4, 2.6, 2.9]
    nt = len(theta)
    flags = (SMERF_RECUR_FP64 if fp64 else 0) | (SMERF_ORDER_PAPER if H == 0 else 0)
    plan = Plan(A=1.0, n_theta=nt, n_phi=n_phi, flags=flags, anchor_spacing=H, khat=list(khat), theta=theta)
    got = plan.sample(6, 2).double().cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle.sample(oracle.KHat(khat), 1.0, nt, n_phi, 6, 2, H=H, theta=theta)
    err = rel_err(got, ref, float(np.std(ref)))
    print("khat at colatitudes %s p=%d fp64=%s: %.2e" % (grid, len(khat), fp64, err))
    assert err < (1e-9 if fp64 else 1e-4)


def test_real_kappa_hat_at_given_colatitudes_is_the_kappa_plan():
    import torch
    from paper_1709_10314_gb300 import Plan
    theta = [0.3, 0.55, 0.9, 1.2, 1.45, 1.7, 2.0]
    a = Plan(A=1.0, n_theta=7, n_phi=32, anchor_spacing=3, khat=[400.0, 2500.0], theta=theta)
    b = Plan([20.0, 50.0], 1.0, 7, 32, anchor_spacing=3, theta=theta)
    assert torch.equal(a.sample(4, 2), b.sample(4, 2))
