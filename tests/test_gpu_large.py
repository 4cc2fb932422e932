"""The large workloads at full size, in the launch configuration bench.py times.

4096 x 8192, C_l = 1/(l(l+1)+100^2), 16 realisations: the precision sweep (recursion FP32 /
FP64 x tables FP32 / FP64) against the oracle on the start ring, and FP32 against FP64
recursion over the whole field.
16384 x 32768, C_l = 1/(l(l+1)+300^2), 4 realisations, FP32 tables: the start ring against
the oracle, sampled bridge tables against Gaussian conditioning, and each sampled ring's
variance against the oracle's exact variance of the discrete field."""
import functools
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

H = 16


@functools.lru_cache(maxsize=None)
def _start_ring(kappa, n_theta, n_phi, seed, n, K, c_diag):
    order = oracle.conditioning_order(n_theta, H)
    return oracle.sample(list(kappa), 1.0, n_theta, n_phi, seed, n, H=H, rings=order[:1], K=K,
                         c_turn_diag=c_diag)[:, 0, :]


SWEEP = {}


@pytest.mark.parametrize("recur,tables", [("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "fp32"), ("fp64", "fp32")])
def test_precision_sweep_4096x8192(recur, tables):
    import torch
    from paper_1709_10314_gb300 import Plan
    from paper_1709_10314_gb300.workloads import flags_for
    kappa, nt, nphi, n = (100.0,), 4096, 8192, 16
    plan = Plan(list(kappa), 1.0, nt, nphi, flags=flags_for(recur, tables), anchor_spacing=H)
    out = plan.sample(1, n)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    k0 = nt // 2
    got = out[[0, n - 1], k0].double().cpu().numpy()
    ref = np.stack([_start_ring(kappa, nt, nphi, 1, 1, 4, 16.0)[0], _start_ring(kappa, nt, nphi, n, 1, 4, 16.0)[0]])
    std = float(np.std(ref))
    err = float(np.max(np.abs(got - ref))) / std
    SWEEP[(recur, tables)] = out[0].double().cpu().numpy() if recur == "fp64" and tables == "fp64" else out[0].cpu()
    print("precision sweep 4096x8192 recur=%s tables=%s: start ring max|gpu-oracle|/std = %.3e" % (recur, tables, err))
    # FP64 throughout: the oracle's own accuracy at K = 4, c_turn_diag = 16 (pinned to 2e-8 of
    # the diagonal scale; measured 1.2e-8); FP64 recursion on FP32 tables: the tables' rounding
    # (measured 1.1e-7); FP32 recursion: 1e-4 of the field std
    bound = {("fp64", "fp64"): 5e-8, ("fp64", "fp32"): 1e-6}.get((recur, tables), 1e-4)
    assert err < bound
    if ("fp64", "fp64") in SWEEP and recur != "fp64":
        ref64 = SWEEP[("fp64", "fp64")]
        e = float(np.max(np.abs(out[0].double().cpu().numpy() - ref64))) / float(np.std(ref64))
        print("  whole field of realisation 0: max|this - FP64/FP64|/std = %.3e" % e)
        assert e < 1e-4


@pytest.fixture(scope="module")
def big():
    import torch
    from paper_1709_10314_gb300 import SMERF_TABLES_FP32, Plan
    plan = Plan([300.0], 1.0, 16384, 32768, flags=SMERF_TABLES_FP32, anchor_spacing=H)
    out = plan.sample(1, 4)
    torch.cuda.synchronize()
    return plan, out


def test_16384x32768_finite_and_start_ring(big):
    import torch
    plan, out = big
    assert out.shape == (4, 16384, 32768)
    assert bool(torch.isfinite(out).all())
    k0 = 8192
    got = out[0, k0].double().cpu().numpy()
    ref = _start_ring((300.0,), 16384, 32768, 1, 1, 5, 8.0)[0]  # oracle same-ring blocks to ~4e-8
    err = float(np.max(np.abs(got - ref))) / float(np.std(ref))
    print("16384x32768 start ring: max|gpu-oracle|/std = %.3e" % err)
    assert err < 1e-4


@pytest.mark.parametrize("m,p", [(0, 3), (4000, 9), (16384, 21)])
def test_16384x32768_sampled_tables(big, m, p):
    plan, _ = big
    nt = 16384
    k0 = nt // 2
    ring, left, right = k0 - p, k0 - p + 1, k0 - (p // H + 1) * H
    th = oracle.ring_theta(nt)[[left, right, ring]]
    S = oracle.cov_m(m, [300.0], 1.0, th)  # full accuracy: rings 2e-4 apart amplify covariance errors
    coef, cov = oracle.conditional_tables(S, 1, 2, [0, 1])
    T = plan.tables(1, 0, p)[:, m]
    half = 0.5 if m > 0 else 1.0
    sd = np.sqrt(np.diag(S))
    assert abs(T[0] - coef[0, 0]) * sd[0] / sd[2] < 1e-5
    assert abs(T[1] - coef[0, 1]) * sd[1] / sd[2] < 1e-5
    assert abs(T[2] ** 2 / half - cov[0, 0]) / sd[2] ** 2 < 1e-5


def test_16384x32768_ring_variance(big):
    """Sample variance of 4 x 32768 points per ring against the exact pointwise variance of
    the m-truncated field, sum_m a_m with a_m = w_m J^m_00 (w = 1, 2, ..., 2, 1/2; Lemma 2.1),
    within 5 sigma.  For a Gaussian ring that is stationary in phi, the mean of T^2 over its
    N points has variance (2/N) sum_d c(d)^2 = 2 (a_0^2 + sum_{0<m<N/2} a_m^2 / 2 + a_{N/2}^2);
    four independent realisations divide it by 4."""
    plan, out = big
    nt, nphi = 16384, 32768
    rings = [8192, 4000]
    # cut-off levels pinned at these rings and orders (tests/test_oracle_cov_high_order.py)
    V = oracle.mode_variances([300.0], 1.0, nt, nphi, K=4, rings=rings, c_turn_diag=4.0)
    w = np.full(nphi // 2 + 1, 2.0)
    w[0], w[-1] = 1.0, 0.5
    for i, k in enumerate(rings):
        a = w * V[:, i]
        exact = float(a.sum())
        x = out[:, k].double().cpu().numpy()
        var = float((x ** 2).mean())
        s2 = 2.0 * (a[0] ** 2 + 0.5 * float((a[1:-1] ** 2).sum()) + a[-1] ** 2) / 4.0
        sig = math.sqrt(s2)
        print("ring %d: sample var %.6e exact %.6e (%.2f sigma)" % (k, var, exact, (var - exact) / sig))
        assert abs(var - exact) < 5 * sig
