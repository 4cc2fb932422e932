"""Allocation failures (SMERF_ENOMEM) through the library's injection hook
(smerf_debug_fail_alloc): plan creation, sampling and batch creation each fail cleanly at every
one of their allocations -- the call returns SMERF_ENOMEM, releases what it had allocated, and
the library keeps working afterwards."""
import pytest

pytestmark = pytest.mark.gpu

ENOMEM = -3


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_plan_creation_fails_cleanly_at_every_allocation():
    from paper_1709_10314_gb300 import Plan, SmerfError, debug_fail_alloc
    Plan([20.0, 50.0], 1.0, 64, 128, anchor_spacing=8).close()  # warm the context and pools
    free0 = _free()
    made_at = None
    for k in range(64):
        debug_fail_alloc(k)
        try:
            plan = Plan([20.0, 50.0], 1.0, 64, 128, anchor_spacing=8)
        except SmerfError as e:
            assert e.status == ENOMEM, (k, e.status)
            continue
        finally:
            debug_fail_alloc(-1)
        made_at = k
        plan.close()
        break
    assert made_at is not None and made_at >= 5, made_at  # a plan makes several allocations
    assert abs(_free() - free0) < (8 << 20)                # nothing was left behind


def test_sampling_and_batches_fail_cleanly_then_recover():
    import torch
    from paper_1709_10314_gb300 import Batch, Plan, SmerfError, debug_fail_alloc
    plan = Plan([10.0], 1.0, 32, 64, anchor_spacing=8)
    ref = plan.sample(5, 3)
    out = torch.full_like(ref, float("nan"))
    debug_fail_alloc(0)  # the call's scratch allocation
    try:
        with pytest.raises(SmerfError) as e:
            plan.sample(5, 3, out)
        assert e.value.status == ENOMEM
    finally:
        debug_fail_alloc(-1)
    torch.cuda.synchronize()
    assert bool(torch.isnan(out).all())  # nothing was launched
    plan.sample(5, 3, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    free0 = _free()
    for k in range(6):
        debug_fail_alloc(k)
        try:
            b = Batch([plan, plan], [2, 1])
        except SmerfError as e:
            assert e.status == ENOMEM
            continue
        finally:
            debug_fail_alloc(-1)
        b.close()
    assert abs(_free() - free0) < (8 << 20)
