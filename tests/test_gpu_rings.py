"""Iso-latitude grids with ring-dependent longitudes (the paper's Sec. 1 remark; HEALPix-like
rings): each ring's point count and offset set by smerf_plan_set_rings, every ring of every
realisation against the oracle's synthesis at the same points (oracle.sample_rings)."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _healpix_like(n_theta, n_phi):
    """Rings of 4 * 2^j points growing towards the equator (at most n_phi), every other ring
    shifted by half a step as HEALPix does."""
    npr, p0 = [], []
    for k in range(n_theta):
        d = min(k, n_theta - 1 - k)  # rings from the nearer pole
        n = 4
        while n < n_phi and n < 4 * (d + 1):
            n *= 2
        npr.append(n)
        p0.append(math.pi / n if k % 2 else 0.0)
    return npr, p0


def _rings(out, npr):
    offs = np.concatenate([[0], np.cumsum(npr)])
    return [[out[j, offs[k]:offs[k + 1]] for k in range(len(npr))] for j in range(out.shape[0])]


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("kappa,n_theta,n_phi,H", [([6.0], 16, 64, 4), ([3.0, 8.0], 12, 32, 0),
                                                 ([2.0, 5.0, 9.0], 14, 64, 3)])
def test_healpix_like_rings_against_oracle(fp64, kappa, n_theta, n_phi, H):
    import torch
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, SMERF_RECUR_FP64, Plan
    flags = (SMERF_RECUR_FP64 if fp64 else 0) | (SMERF_ORDER_PAPER if H == 0 else 0)
    plan = Plan(kappa, 1.0, n_theta, n_phi, flags=flags, anchor_spacing=H)
    npr, p0 = _healpix_like(n_theta, n_phi)
    plan.set_rings(npr, p0)
    assert plan.info()["points_per_sample"] == sum(npr)
    out = plan.sample(21, 3)
    torch.cuda.synchronize()
    assert tuple(out.shape) == (3, sum(npr))
    got = _rings(out.double().cpu().numpy(), npr)
    ref = oracle.sample_rings(kappa, 1.0, n_theta, npr, p0, 21, 3, H=H, n_phi=n_phi)
    std = float(np.std(np.concatenate([np.concatenate(r) for r in ref])))
    err = max(float(np.max(np.abs(got[j][k] - ref[j][k]))) for j in range(3) for k in range(n_theta)) / std
    print("rings %s fp64=%s: max|gpu-oracle|/std = %.2e" % (npr, fp64, err))
    assert err < (1e-9 if fp64 else 1e-4)


def test_full_rings_and_reset():
    """Full rings without offsets reproduce the plain grid bit for bit; offsets only shift the
    points; set_rings(None) restores the plain grid."""
    import torch
    from paper_1709_10314_gb300 import Plan
    plan = Plan([20.0, 50.0], 1.0, 32, 128, anchor_spacing=8)
    ref = plan.sample(4, 2)
    plan.set_rings([128] * 32)
    full = plan.sample(4, 2)
    torch.cuda.synchronize()
    assert torch.equal(full.reshape(ref.shape), ref)
    shift = [(3 * k) % 128 for k in range(32)]
    plan.set_rings([128] * 32, [2 * math.pi * s / 128 for s in shift])
    sh = plan.sample(4, 2).reshape(ref.shape)
    torch.cuda.synchronize()
    for k in range(32):
        d = float((sh[:, k] - torch.roll(ref[:, k], -shift[k], dims=1)).abs().max())
        assert d <= 1e-4 * float(ref.std())
    plan.set_rings(None)
    assert torch.equal(plan.sample(4, 2), ref)


def test_ring_layout_rejections():
    import torch
    from paper_1709_10314_gb300 import SMERF_TABLES_FP32, Plan, SmerfError
    plan = Plan([10.0], 1.0, 8, 32, anchor_spacing=4)
    for bad in ([13] * 8, [2] * 8, [64] * 8):  # odd, fewer than 4, more than n_phi
        with pytest.raises(SmerfError) as e:
            plan.set_rings(bad)
        assert e.value.status == -1
    big = Plan([300.0], 1.0, 4, 32768, flags=SMERF_TABLES_FP32)  # the ring kernel's size
    with pytest.raises(SmerfError) as e:
        big.set_rings([32768, 16384, 16384, 32768])
    assert e.value.status == -5
    torch.cuda.synchronize()


def test_ring_plans_in_a_batch():
    """A batch launches the requests of ring-dependent plans individually, beside its batched
    groups; every request's output equals the single call's, bit for bit, in both launch forms."""
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, Batch, Plan, sample_batched
    a = Plan([6.0], 1.0, 16, 64, anchor_spacing=4)
    b = Plan([3.0, 8.0], 1.0, 12, 32, flags=SMERF_RECUR_FP64, anchor_spacing=4)
    c = Plan([10.0], 1.0, 32, 64, anchor_spacing=8)  # plain grid: batched
    for pl, (nt, nphi) in ((a, (16, 64)), (b, (12, 32))):
        npr, p0 = _healpix_like(nt, nphi)
        pl.set_rings(npr, p0)
    plans, counts, seeds = [a, b, c], [3, 2, 2], [7, 8, 9]
    ref = [p.sample(s, n) for p, s, n in zip(plans, seeds, counts)]
    bt = Batch(plans, counts)
    assert bt.info()["singles"] == 2 and bt.info()["groups"] == 1
    for single in (False, True):
        bt.set_single_launch(single)
        outs = [torch.full_like(r, float("nan")) for r in ref]
        bt.sample(seeds, outs)
        assert bt.status() == 0
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
    outs = [torch.full_like(r, float("nan")) for r in ref]
    sample_batched(plans, seeds, counts, outs)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    # the C ABI cannot see a buffer's length: the binding checks it against the ring layout
    short = [o[:, :-1].contiguous() if i == 0 else o for i, o in enumerate(outs)]
    with pytest.raises(ValueError):
        bt.sample(seeds, short)
    bt.close()


def _healpix(nside):
    """HEALPix rings (colatitudes, point counts, first-pixel longitudes), the pixelisation's
    published formulae (Gorski et al. 2005), as in the oracle's own HEALPix tests."""
    from test_oracle_healpix import healpix_rings
    return healpix_rings(nside)


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("nside,n_phi,kappa,H", [(3, 16, [3.0, 7.0], 0), (4, 16, [6.0], 4),
                                                 (6, 32, [5.0, 12.0], 5), (3, 16, [2.0, 5.0, 9.0], 3)])
def test_healpix_grid_against_oracle(fp64, nside, n_phi, kappa, H):
    """Full HEALPix grids: rings at the HEALPix colatitudes (smerf_plan_create_theta) with 4i
    points in the polar caps and 4 nside in the belt, half-pixel offsets as HEALPix places them
    (smerf_plan_set_rings; 12-, 20- and 24-point rings take the direct synthesis), every ring of
    every realisation against the oracle at the same points."""
    import torch
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, SMERF_RECUR_FP64, Plan
    th, npr, p0 = _healpix(nside)
    nt = len(th)
    flags = (SMERF_RECUR_FP64 if fp64 else 0) | (SMERF_ORDER_PAPER if H == 0 else 0)
    plan = Plan(kappa, 1.0, nt, n_phi, flags=flags, anchor_spacing=H, theta=list(th))
    plan.set_rings(npr, p0)
    assert plan.info()["points_per_sample"] == 12 * nside * nside
    out = plan.sample(31, 2)
    torch.cuda.synchronize()
    got = _rings(out.double().cpu().numpy(), npr)
    ref = oracle.sample_rings(kappa, 1.0, nt, npr, p0, 31, 2, H=H, n_phi=n_phi, theta=th)
    std = float(np.std(np.concatenate([np.concatenate(r) for r in ref])))
    err = max(float(np.max(np.abs(got[j][k] - ref[j][k]))) for j in range(2) for k in range(nt)) / std
    print("HEALPix nside %d p=%d fp64=%s: max|gpu-oracle|/std = %.2e" % (nside, len(kappa), fp64, err))
    assert err < (1e-9 if fp64 else 1e-4)


def test_colatitudes_given_explicitly_are_the_default_grid():
    """The equiangular colatitudes passed to smerf_plan_create_theta build the same tables as the
    default plan: the same field bit for bit."""
    import torch
    from paper_1709_10314_gb300 import Plan
    th = oracle.ring_theta(24)
    a = Plan([20.0, 50.0], 1.0, 24, 64, anchor_spacing=6).sample(5, 3)
    b = Plan([20.0, 50.0], 1.0, 24, 64, anchor_spacing=6, theta=list(th)).sample(5, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def _band(lo, hi, n, seed):
    """n increasing colatitudes from lo to hi with uneven steps."""
    w = 1.0 + 0.6 * np.random.default_rng(seed).random(n - 1)
    return list(lo + (hi - lo) * np.concatenate([[0.0], np.cumsum(w) / w.sum()]))


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("kappa,theta,n_phi,H", [
    ([6.0], _band(0.2, 1.4, 12, 1), 32, 4),               # northern band: the southern chain is empty
    ([3.0, 8.0], _band(0.4, 2.9, 15, 2), 64, 0),          # straddling the equator, Alg. 2's order
    ([2.0, 5.0, 9.0], _band(1.9, 2.9, 10, 3), 32, 3),     # southern band: the northern chain is empty
    ([20.0], _band(0.3, 1.5, 9, 4) + _band(1.7, 2.0, 4, 5), 256, 3),      # start ring north of the
    ([20.0, 45.0], _band(0.3, 1.5, 9, 4) + _band(1.7, 2.0, 4, 5), 256, 0),  # equator, many modes
    ([20.0, 45.0], _band(1.0, 1.45, 5, 6) + _band(1.62, 2.8, 9, 7), 256, 4),  # ... south of it
])
def test_band_grid_against_oracle(fp64, kappa, theta, n_phi, H):
    """Grids that are not symmetric about the equator (a band of latitudes, or rings placed
    unevenly about the equator; the Sec. 1 remark that any iso-latitude grid serves): the chains
    start at the ring nearest the equator and the southern chain's steps are computed on their
    own; every ring of every realisation against the oracle on the same colatitudes."""
    import torch
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, SMERF_RECUR_FP64, Plan
    nt = len(theta)
    flags = (SMERF_RECUR_FP64 if fp64 else 0) | (SMERF_ORDER_PAPER if H == 0 else 0)
    plan = Plan(kappa, 1.0, nt, n_phi, flags=flags, anchor_spacing=H, theta=theta)
    out = plan.sample(17, 2)
    torch.cuda.synchronize()
    ref = oracle.sample(kappa, 1.0, nt, n_phi, 17, 2, H=H, theta=theta)
    err = float(np.max(np.abs(out.double().cpu().numpy() - ref))) / float(np.std(ref))
    print("band k0=%d p=%d fp64=%s: max|gpu-oracle|/std = %.2e" % (
        oracle.start_ring(nt, theta), len(kappa), fp64, err))
    assert err < (1e-9 if fp64 else 1e-4)


def test_colatitude_rejections():
    from paper_1709_10314_gb300 import Plan, SmerfError
    th = list(oracle.ring_theta(8))
    for bad in (th[::-1], th[:-1] + [math.pi], [0.0] + th[1:], th[:4] + th[3:7]):
        with pytest.raises(SmerfError) as e:
            Plan([10.0], 1.0, 8, 32, theta=bad)
        assert e.value.status == -1
