"""Three spectrum factors, p = 3 (Eq. (Cl) with three kappa_i: a 3-vector state per real
chain, Eqs. (trans_matrix), (innov_matrix), (state_space)).  The CUDA path through the C ABI
against the oracle on the same seeded inputs, element by element: FP64 recursion within 1e-10
of the field std on small grids in both orders, FP32 recursion within 1e-4; the launch
candidates (one to eight units per producer thread) with the built-in FFT radix plan bit for bit
against the built-in choice, the other radix plan to rounding; batches holding p = 3 requests
against single calls."""
import numpy as np
import pytest

import oracle
from gpu_util import oracle_field, oracle_std, rel_err

pytestmark = pytest.mark.gpu

K3 = (4.0, 9.0, 20.0)


def _plan(n_theta, n_phi, H, flags=0, kappa=K3):
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, Plan
    if H == 0:
        flags |= SMERF_ORDER_PAPER
    return Plan(list(kappa), 1.0, n_theta, n_phi, flags=flags, anchor_spacing=H)


@pytest.mark.parametrize("n_theta,n_phi,H,n", [(20, 64, 0, 2), (21, 64, 6, 3), (16, 128, 5, 1)])
def test_fp64_small_grids(n_theta, n_phi, H, n):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    plan = _plan(n_theta, n_phi, H, SMERF_RECUR_FP64)
    assert plan.info()["p"] == 3
    got = plan.sample(21, n).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle_field(K3, 1.0, n_theta, n_phi, 21, n, H)
    err = rel_err(got, ref, oracle_std(K3, 1.0, n_theta, n_phi))
    print("p = 3 FP64 %d x %d H=%d: max|gpu-oracle|/std = %.2e" % (n_theta, n_phi, H, err))
    assert got.dtype == np.float64 and err < 1e-10


@pytest.mark.parametrize("n_theta,n_phi,H,n,seed", [
    (20, 64, 0, 2, 5),          # Alg. 2's order
    (21, 64, 6, 5, 6),          # odd n_theta, anchors and bridges
    (9, 512, 4, 3, 7),          # several warps of producers
    (12, 8, 3, 1, 2**64 - 1),   # smallest n_phi; the key wraps for no realisation here
])
def test_fp32_small_grids(n_theta, n_phi, H, n, seed):
    import torch
    plan = _plan(n_theta, n_phi, H)
    got = plan.sample(seed, n).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle_field(K3, 1.0, n_theta, n_phi, seed, n, H)
    err = rel_err(got, ref, float(np.std(ref)))
    print("p = 3 FP32 %d x %d H=%d: max|gpu-oracle|/std = %.2e" % (n_theta, n_phi, H, err))
    assert got.dtype == np.float32 and np.all(np.isfinite(got)) and err < 1e-4


def test_fp64_tables_fp32_recursion_staged_and_in_kernel():
    """FP64 tables with FP32 recursion: five realisations stage the tables as FP32 once per
    call, two convert them inside the kernels; both use the same truncating conversion, so the
    common realisations are identical, and both match the oracle."""
    import torch
    from paper_1709_10314_gb300 import SMERF_TABLES_FP64
    plan = _plan(21, 64, 6, SMERF_TABLES_FP64)
    five = plan.sample(9, 5)
    two = plan.sample(9, 2)
    torch.cuda.synchronize()
    assert torch.equal(five[:2], two)
    ref = oracle_field(K3, 1.0, 21, 64, 9, 5, 6)
    assert rel_err(five.cpu().numpy(), ref, float(np.std(ref))) < 1e-4


@pytest.mark.parametrize("n_theta,n_phi,H,n", [(6, 4096, 2, 2), (4, 8192, 0, 1)])
def test_fp32_long_rings_every_candidate(n_theta, n_phi, H, n):
    """Rings of 2048 and 4096 complex points (two and four units per producer thread in the
    built-in launch; the candidates take two to eight): the built-in choice against the oracle (spectral sums at K = 4,
    c_turn_diag = 8, pinned at these orders to 3e-6 of the diagonal scale), every other launch
    candidate bit for bit against it."""
    import torch
    plan = _plan(n_theta, n_phi, H)
    ref_gpu = plan.sample(13, n)
    torch.cuda.synchronize()
    ref = oracle.sample(list(K3), 1.0, n_theta, n_phi, 13, n, H=H, K=4, c_turn_diag=8.0)
    err = rel_err(ref_gpu.cpu().numpy(), ref, float(np.std(ref)))
    print("p = 3 FP32 %d x %d H=%d: max|gpu-oracle|/std = %.2e" % (n_theta, n_phi, H, err))
    assert err < 1e-4
    cands = plan.launch_candidates()
    assert len(cands) >= 2
    for cfg in cands:
        plan.set_launch(cfg)
        got = plan.sample(13, n)
        torch.cuda.synchronize()
        if cfg[5] == 16:   # the built-in radix plan
            assert torch.equal(got, ref_gpu), cfg
        else:
            assert rel_err(got.cpu().numpy(), ref, float(np.std(ref))) < 1e-4, cfg
    plan.set_launch(None)


@pytest.mark.parametrize("flags_name", ["fp32", "fp64"])
def test_every_candidate_gives_the_same_field(flags_name):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    plan = _plan(24, 512, 5, SMERF_RECUR_FP64 if flags_name == "fp64" else 0)
    ref = plan.sample(4, 3)
    torch.cuda.synchronize()
    cands = plan.launch_candidates()
    assert len(cands) >= 2 and all(c[1] == 1 and c[4] == 1 for c in cands)
    default_radix = 4 if flags_name == "fp64" else 16
    for cfg in cands:
        plan.set_launch(cfg)
        got = plan.sample(4, 3)
        if cfg[5] == default_radix:
            assert torch.equal(got, ref), cfg
        else:
            assert float((got.double() - ref.double()).abs().max() / ref.double().std()) < 1e-5, cfg
    plan.set_launch(None)


def test_batch_with_p3_requests_equals_single_calls():
    """p = 3 requests run in a batch as one anchor and one segment launch per kernel shape,
    beside the anchor and persistent launches of the p = 1, 2 requests."""
    import torch
    from paper_1709_10314_gb300 import Batch, SMERF_RECUR_FP64
    plans = [_plan(24, 512, 5), _plan(17, 256, 4), _plan(24, 512, 5, kappa=(6.0,)),
             _plan(16, 128, 4, kappa=(5.0, 11.0)), _plan(16, 128, 4, SMERF_RECUR_FP64)]
    counts = [2, 3, 2, 1, 2]
    seeds = [101, 202, 303, 404, 505]
    outs = [torch.empty((n, p.n_theta, p.n_phi), dtype=torch.float64 if i == 4 else torch.float32,
                        device="cuda") for i, (p, n) in enumerate(zip(plans, counts))]
    b = Batch(plans, counts)
    b.sample(seeds, outs)
    torch.cuda.synchronize()
    for p, n, s, o in zip(plans, counts, seeds, outs):
        assert torch.equal(o, p.sample(s, n))
    # an anchor and a persistent launch (p = 1, 2), a launch pair for each p = 3 shape: 24 x 512
    # and 17 x 256 in FP32, 16 x 128 in FP64
    assert b.info()["launches"] == 2 + 2 * 3


def test_p3_too_long_rings_rejected():
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SmerfError
    with pytest.raises(SmerfError) as e:
        _plan(8, 16384, 4)
    assert e.value.status == -5
    with pytest.raises(SmerfError) as e:
        _plan(8, 8192, 4, SMERF_RECUR_FP64)
    assert e.value.status == -5
