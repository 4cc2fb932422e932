"""smerf_sample_noalloc, the entry point for callers that cannot let the library allocate
device memory (graphs captured once and replayed, pre-carved device memory, frameworks
that own every device byte).  Its output must equal smerf_sample's on the same plan and
seeds, call after call, since both run the same kernels; only the scratch location
differs (a fixed 16 MiB device array instead of the stream-ordered allocator).

Named test_zz_* so that pytest collects it last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp64", [False, True])
def test_noalloc_matches_allocating_entry_twice(fp64):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, Plan
    plan = Plan([10.0], 1.0, 32, 64, flags=SMERF_RECUR_FP64 if fp64 else 0, anchor_spacing=8)
    tol = 1e-10 if fp64 else 1e-4
    for seed, n in [(3, 5), (11, 2)]:  # two calls in a row reuse the same fixed scratch
        ref = plan.sample(seed, n)
        got = torch.full_like(ref, float("nan"))
        plan.sample_noalloc(seed, n, got)
        torch.cuda.synchronize()
        r = ref.double().cpu().numpy()
        g = got.double().cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) / float(np.std(r)) <= tol


def test_noalloc_p2_grid_and_rejects_oversize():
    import torch
    from paper_1709_10314_gb300 import Plan, SmerfError
    plan = Plan([20.0, 50.0], 1.0, 64, 128, anchor_spacing=8)
    ref = plan.sample(7, 4)
    got = torch.empty_like(ref)
    plan.sample_noalloc(7, 4, got)
    torch.cuda.synchronize()
    assert float((got - ref).abs().max()) / float(ref.std()) <= 1e-4
    per = plan.info()["scratch_bytes_per_sample"]
    n_big = (16 << 20) // per + 1
    with pytest.raises(SmerfError) as e:
        plan.sample_noalloc(1, n_big, torch.empty((n_big, 64, 128), dtype=torch.float32, device="cuda"))
    assert e.value.status == -6
