"""Field parity: the CUDA path through the C ABI against the oracle, element by element
on the same seeded inputs.  FP64 recursion: within 1e-10 of the field std; FP32
recursion: within 1e-4 of the field std."""
import numpy as np
import pytest

import oracle
from gpu_util import oracle_field, oracle_std, rel_err

pytestmark = pytest.mark.gpu


def _plan(kappa, n_theta, n_phi, H, flags=0, A=1.0):
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, Plan
    if H == 0:
        flags |= SMERF_ORDER_PAPER
    return Plan(kappa, A, n_theta, n_phi, flags=flags, anchor_spacing=H)


@pytest.mark.parametrize("H", [0, 32, 7])
def test_fp64_plain_method_64x128(H):
    """The plain-method FP64 case: 64 x 128 grid, C_l = 1/(l(l+1)+100), seed 1."""
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    plan = _plan([10.0], 64, 128, H, SMERF_RECUR_FP64)
    got = plan.sample(1, 1).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle_field((10.0,), 1.0, 64, 128, 1, 1, H)
    std = oracle_std((10.0,), 1.0, 64, 128)
    assert got.dtype == np.float64 and got.shape == (1, 64, 128)
    assert rel_err(got, ref, std) < 1e-10


@pytest.mark.parametrize("kappa,n_theta,n_phi,H,n,seed", [
    ((10.0,), 32, 64, 8, 5, 11),          # ragged realisation groups (5 = 4 + 1)
    ((3.0, 8.0), 33, 64, 4, 3, 2),        # odd n_theta: start on the equator ring
    ((20.0, 50.0), 16, 32, 0, 2, 7),      # Alg. 2's order, p = 2
    ((5.0,), 40, 256, 6, 9, 123),         # several tiles of slots, last segment short
    ((2.0, 7.0), 24, 8, 5, 1, 2**64 - 1), # smallest n_phi; key wraps to 0 for no realisation here
])
def test_fp32_small_grids(kappa, n_theta, n_phi, H, n, seed):
    import torch
    plan = _plan(list(kappa), n_theta, n_phi, H)
    got = plan.sample(seed, n).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle_field(kappa, 1.0, n_theta, n_phi, seed, n, H)
    std = float(np.std(ref))
    assert got.dtype == np.float32
    assert np.all(np.isfinite(got))
    assert rel_err(got, ref, std) < 1e-4


@pytest.mark.parametrize("flags_name", ["fp32_rec_fp64_tab", "fp64_rec_fp32_tab"])
def test_mixed_precision(flags_name):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_TABLES_FP32, SMERF_TABLES_FP64
    flags = SMERF_TABLES_FP64 if flags_name == "fp32_rec_fp64_tab" else (SMERF_RECUR_FP64 | SMERF_TABLES_FP32)
    plan = _plan([10.0], 32, 64, 8, flags)
    got = plan.sample(3, 2).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle_field((10.0,), 1.0, 32, 64, 3, 2, 8)
    assert rel_err(got, ref, float(np.std(ref))) < 1e-4


@pytest.mark.parametrize("n_theta", [2, 3, 4])
def test_tiny_grids(n_theta):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    plan = _plan([4.0], n_theta, 8, 0, SMERF_RECUR_FP64)
    got = plan.sample(5, 3).cpu().numpy()
    torch.cuda.synchronize()
    ref = oracle_field((4.0,), 1.0, n_theta, 8, 5, 3, 0)
    assert rel_err(got, ref, float(np.std(ref))) < 1e-10


def test_zero_samples_and_amplitude():
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, Plan
    plan = Plan([4.0], 2.5, 8, 16, flags=SMERF_RECUR_FP64, anchor_spacing=2)
    out = torch.full((1, 8, 16), 7.0, dtype=torch.float64, device="cuda")
    plan.sample(1, 0, out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    got = plan.sample(9, 1).cpu().numpy()
    ref = oracle.sample([4.0], 2.5, 8, 16, 9, 1, H=2)
    assert rel_err(got, ref, float(np.std(ref))) < 1e-10


def test_host_entry_matches_device():
    import torch
    plan = _plan([10.0], 32, 64, 8)
    dev = plan.sample(42, 3).cpu().numpy()
    host = plan.sample_host(42, 3)
    torch.cuda.synchronize()
    assert np.array_equal(dev, host)


def test_host_entry_pinned_memory_written_directly():
    # page-locked host output: the kernels write it over the CPU-GPU link; same field, twice
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64
    for flags, dt in ((0, torch.float32), (SMERF_RECUR_FP64, torch.float64)):
        plan = _plan([20.0, 50.0], 64, 256, 16, flags)
        dev = plan.sample(7, 5).cpu()
        pinned = torch.full((5, 64, 256), float("nan"), dtype=dt, pin_memory=True)
        for _ in range(2):
            plan.sample_host(7, 5, pinned)
            assert torch.equal(pinned, dev)


def test_batched_matches_single_calls():
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, sample_batched
    p1 = _plan([10.0], 32, 64, 8)
    p2 = _plan([3.0, 8.0], 17, 32, 4, SMERF_RECUR_FP64)
    o1 = torch.empty((3, 32, 64), dtype=torch.float32, device="cuda")
    o2 = torch.empty((2, 17, 32), dtype=torch.float64, device="cuda")
    sample_batched([p1, p2], [5, 6], [3, 2], [o1, o2])
    torch.cuda.synchronize()
    assert torch.equal(o1, p1.sample(5, 3))
    assert torch.equal(o2, p2.sample(6, 2))


def test_staged_fp64_tables_equal_in_kernel_conversion():
    # FP64 tables with FP32 recursion: a call with several realisations converts the tables to
    # FP32 once (staged); a batched launch converts them in the kernels.  Same field, bit for bit.
    import torch
    from paper_1709_10314_gb300 import SMERF_TABLES_FP64, sample_batched
    for kappa, nt, nphi, H in (([20.0, 50.0], 40, 128, 8), ([30.0], 33, 64, 4)):
        plan = _plan(kappa, nt, nphi, H, SMERF_TABLES_FP64)
        # staged: a short conversion launch ahead of the anchor (which converts the step
        # tables) and segment launches
        assert (plan.launches(6), plan.launches(3), plan.launches(0)) == (3, 2, 0)
        staged = plan.sample(5, 6)
        out = torch.empty_like(staged)
        sample_batched([plan], [5], [6], [out])
        torch.cuda.synchronize()
        assert torch.equal(staged, out)


def test_scratch_pool_kept_and_trimmed_between_calls():
    # per-call scratch comes from the library's pool; trimming it between calls changes nothing
    import torch
    from paper_1709_10314_gb300 import SMERF_TABLES_FP64, last_device_status, scratch_trim
    plan = _plan([20.0, 50.0], 40, 128, 8, SMERF_TABLES_FP64)
    a = plan.sample(3, 6)
    assert last_device_status() == 0
    scratch_trim()
    b = plan.sample(3, 6)
    host = plan.sample_host(3, 6)
    torch.cuda.synchronize()
    scratch_trim()
    assert torch.equal(a, b)
    assert np.array_equal(a.cpu().numpy(), host)


def test_plans_created_together_equal_plans_created_one_by_one():
    # smerf_plan_create_many overlaps the set-ups on several streams: the same tables, bit for bit
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_TABLES_FP64, Plan, SmerfError, create_plans
    specs = [dict(kappa=[10.0], n_theta=32, n_phi=64, anchor_spacing=8),
             dict(kappa=[3.0, 8.0], n_theta=33, n_phi=64, anchor_spacing=4, flags=SMERF_RECUR_FP64),
             dict(kappa=[20.0, 50.0], n_theta=64, n_phi=256, anchor_spacing=16, flags=SMERF_TABLES_FP64),
             dict(kappa=[150.0], n_theta=128, n_phi=256, anchor_spacing=0)] * 5
    many = create_plans(specs)
    assert len(many) == len(specs)
    for d, pm in zip(specs, many):
        p1 = Plan(d["kappa"], 1.0, d["n_theta"], d["n_phi"], flags=d.get("flags", 0),
                  anchor_spacing=d.get("anchor_spacing", 0))
        for kind, c, pos in ((0, 0, 0), (1, 0, 1), (1, 1, 2), (2, 0, 1)):
            try:
                a, b = p1.tables(kind, c, pos), pm.tables(kind, c, pos)
            except SmerfError:  # no coarse rows without anchors
                continue
            assert np.array_equal(a, b)
        assert torch.equal(p1.sample(9, 2), pm.sample(9, 2))
