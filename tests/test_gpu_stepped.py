"""Stepped rings of the tuned kernel builds against the oracle (Eq. (state_space), Alg. 2).

The full-size workloads can only afford the oracle on their start ring; these cases run the
same kernel instantiations and launch configurations on grids where the oracle reaches the
rings that the recursion steps:

* 1024 x 2048, p = 2, Alg. 2's order (no anchors): the first band of the northern chain
  (the start ring and the next 7 rings), in the launch configurations bench.py uses for the
  1024 x 2048 workload (FP32 recursion with FP64 tables staged as FP32 and with FP32 tables;
  FP64 recursion);
* 48 x 2048, p = 2, anchors every 16 rings: the start ring, both anchors and the whole first
  northern segment, whose rings are bridges conditioned on the left neighbour and the right
  anchor, in the same FP32 launch configuration;
* 4 x 32768, p = 1, Alg. 2's order: the start ring and the ring stepped from it, through the
  ring kernel that the 16384 x 32768 workload runs (16384-point FFT, 8 units per thread);
* 24 x 16384, p = 1, anchors every 8 rings: the start ring, both anchors and the first three
  bridge rings, through the ring kernel's 8192-point build with its right-anchor term.

Oracle cut-off levels other than the defaults are pinned at these rings and orders in
tests/test_oracle_cov_high_order.py."""
import numpy as np
import pytest

import oracle
from gpu_util import oracle_field, rel_err

pytestmark = pytest.mark.gpu

KAPPA2 = (20.0, 50.0)
C2_LAUNCH = {("fp32", "fp64"): (4, 1, 256, 64, 2, 16), ("fp32", "fp32"): (4, 1, 256, 64, 2, 16),
             ("fp64", "fp64"): (4, 1, 256, 128, 1, 4)}


def _plan(kappa, nt, nphi, recur, tables, H, launch=None):
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, Plan
    from paper_1709_10314_gb300.workloads import flags_for
    flags = flags_for(recur, tables) | (SMERF_ORDER_PAPER if H == 0 else 0)
    plan = Plan(list(kappa), 1.0, nt, nphi, flags=flags, anchor_spacing=H)
    if launch is not None:
        assert tuple(launch) in plan.launch_candidates()
        plan.set_launch(launch)
    return plan


@pytest.mark.parametrize("recur,tables", [("fp32", "fp64"), ("fp32", "fp32"), ("fp64", "fp64")])
def test_first_band_1024x2048_alg2_order(recur, tables):
    import torch
    nt, nphi, n, h = 1024, 2048, 4, 8
    plan = _plan(KAPPA2, nt, nphi, recur, tables, 0, C2_LAUNCH[(recur, tables)])
    out = plan.sample(7, n)
    torch.cuda.synchronize()
    rings = tuple(oracle.conditioning_order(nt, 0)[:h])
    assert rings == tuple(range(512, 504, -1))
    ref = oracle_field(KAPPA2, 1.0, nt, nphi, 7, n, 0, rings)
    got = out[:, list(rings)].double().cpu().numpy()
    err = rel_err(got, ref, float(np.std(ref)))
    print("1024x2048 Alg. 2 order, rings 512..505, recur=%s tables=%s: max|gpu-oracle|/std = %.2e" % (recur, tables, err))
    # FP64: the oracle's dense factor of eight rings pi/1024 apart loses digits to the
    # near-singular joint covariance (innovations ~ dtheta^3 of the marginal, p = 2)
    assert err < (1e-8 if recur == "fp64" else 1e-4)


def test_first_segment_48x2048_anchored():
    """Every ring of the first northern segment is a bridge between its left neighbour and the
    anchor 16 rings out (right-anchor term C x_anchor); FP64 tables staged as FP32 (4
    realisations), the 1024 x 2048 workload's FP32 launch configuration."""
    import torch
    nt, nphi, n, H = 48, 2048, 4, 16
    plan = _plan(KAPPA2, nt, nphi, "fp32", "fp64", H, C2_LAUNCH[("fp32", "fp64")])
    out = plan.sample(11, n)
    torch.cuda.synchronize()
    order = oracle.conditioning_order(nt, H)
    rings = tuple(order[:18])
    assert rings[:3] == (24, 8, 40) and rings[3:] == tuple(range(23, 8, -1))
    ref = oracle.sample(list(KAPPA2), 1.0, nt, nphi, 11, n, H=H, rings=list(rings), K=4, c_turn_diag=8.0)
    got = out[:, list(rings)].double().cpu().numpy()
    err = rel_err(got, ref, float(np.std(ref)))
    print("48x2048 anchored, start ring, anchors and first segment: max|gpu-oracle|/std = %.2e" % err)
    assert err < 1e-4


def test_stepped_ring_32768_inplace_kernel():
    """The ring kernel of the 16384 x 32768 workload (p = 1, 16384-point FFT, 8 units per
    thread, states of 6 parked in shared memory) on a 4-ring grid: start ring and the ring the
    recursion steps from it."""
    import torch
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, SMERF_TABLES_FP32, Plan
    nt, nphi, n = 4, 32768, 2
    plan = Plan([300.0], 1.0, nt, nphi, flags=SMERF_TABLES_FP32 | SMERF_ORDER_PAPER, anchor_spacing=0)
    assert plan.launch_candidates() == []  # no warp-specialised build: the in-place kernel runs
    out = plan.sample(5, n)
    torch.cuda.synchronize()
    rings = oracle.conditioning_order(nt, 0)[:2]
    assert rings == [2, 1]
    ref = oracle.sample([300.0], 1.0, nt, nphi, 5, n, H=0, rings=rings, K=4, c_turn_diag=4.0)
    got = out[:, rings].double().cpu().numpy()
    err = rel_err(got, ref, float(np.std(ref)))
    print("4x32768 Alg. 2 order, rings 2 and 1: max|gpu-oracle|/std = %.2e" % err)
    assert err < 1e-4


def test_bridge_rings_16384_ring_kernel():
    """The ring kernel's 8192-point build (two CTAs per SM) with right anchors: rings 11, 10, 9
    are bridges between the start ring 12 and the anchor 4."""
    import torch
    from paper_1709_10314_gb300 import SMERF_TABLES_FP32, Plan
    nt, nphi, n, H = 24, 16384, 2, 8
    plan = Plan([300.0], 1.0, nt, nphi, flags=SMERF_TABLES_FP32, anchor_spacing=H)
    out = plan.sample(3, n)
    torch.cuda.synchronize()
    rings = oracle.conditioning_order(nt, H)[:6]
    assert rings == [12, 4, 20, 11, 10, 9]
    ref = oracle.sample([300.0], 1.0, nt, nphi, 3, n, H=H, rings=rings, K=4, c_turn_diag=4.0)
    got = out[:, rings].double().cpu().numpy()
    err = rel_err(got, ref, float(np.std(ref)))
    print("24x16384 anchored, start ring, anchors, bridge rings 11..9: max|gpu-oracle|/std = %.2e" % err)
    assert err < 1e-4
