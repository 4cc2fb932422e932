"""The bench workload at full size (1024 x 2048, C_l = 1/((l(l+1)+20^2)(l(l+1)+50^2)),
64 realisations, FP64 tables, FP32 recursion + FFT, anchors every 16 rings), in the
launch configuration bench.py times.  The oracle computes sampled outputs it can
afford: the start ring of realisations 0 and 63, and sampled table entries by Gaussian
conditioning on a few rings; properties that hold at any size cover the rest."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

KAPPA, A, NT, NP, NS, H = [20.0, 50.0], 1.0, 1024, 2048, 64, 16


@pytest.fixture(scope="module")
def fields():
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_TABLES_FP64, Plan
    plan32 = Plan(KAPPA, A, NT, NP, flags=SMERF_TABLES_FP64, anchor_spacing=H)
    out = plan32.sample(1, NS)
    plan64 = Plan(KAPPA, A, NT, NP, flags=SMERF_RECUR_FP64, anchor_spacing=H)
    out64 = plan64.sample(1, 2)
    torch.cuda.synchronize()
    return plan32, out, out64


def test_finite_and_shape(fields):
    plan, out, _ = fields
    import torch
    assert out.shape == (NS, NT, NP) and out.dtype == torch.float32
    assert bool(torch.isfinite(out).all())


def test_start_ring_against_oracle(fields):
    plan, out, _ = fields
    order = oracle.conditioning_order(NT, H)
    k0 = order[0]
    ref = oracle.sample(KAPPA, A, NT, NP, 1, 1, H=H, rings=order[:1])[0, 0]
    ref63 = oracle.sample(KAPPA, A, NT, NP, 1 + 63, 1, H=H, rings=order[:1])[0, 0]
    std = float(np.std(ref))
    got = out[0, k0].cpu().numpy().astype(np.float64)
    got63 = out[63, k0].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) / std < 1e-4
    assert np.max(np.abs(got63 - ref63)) / std < 1e-4


def test_fp32_within_tolerance_of_fp64(fields):
    _, out, out64 = fields
    a = out[:2].double().cpu().numpy()
    b = out64.cpu().numpy()
    std = float(np.std(b))
    assert np.max(np.abs(a - b)) / std < 1e-4


@pytest.mark.parametrize("m,p", [(0, 1), (3, 5), (517, 17), (1024, 15), (200, 33)])
def test_sampled_tables(fields, m, p):
    """Bridge table at chain position p (north) for mode m against conditioning on
    (left neighbour, right anchor) in the spectral-sum covariance of three rings."""
    from paper_1709_10314_gb300 import SMERF_TABLES_FP64, Plan
    plan, _, _ = fields
    k0 = NT // 2
    ring, left = k0 - p, k0 - p + 1
    right = k0 - (p // H + 1) * H
    rings = [left, right, ring]
    th = oracle.ring_theta(NT)[rings]
    S = oracle.cov_m(m, KAPPA, A, th, K=4)
    M = 2
    coef, cov = oracle.conditional_tables(S, M, 2, [0, 1])
    T = plan.tables(1, 0, p)[:, m]
    Ag, Cg = T[:4].reshape(2, 2), T[4:8].reshape(2, 2)
    Bg = np.array([[T[8], 0.0], [T[9], T[10]]])
    half = 0.5 if m > 0 else 1.0
    sd = np.sqrt(np.diag(S)).reshape(3, 2)
    for blk, par in [(Ag, 0), (Cg, 1)]:
        err = np.abs(blk - coef[:, 2 * par:2 * par + 2]) * sd[par][None, :] / sd[2][:, None]
        assert err.max() < 1e-6
    err = np.abs(Bg @ Bg.T / half - cov) / np.outer(sd[2], sd[2])
    assert err.max() < 1e-6
