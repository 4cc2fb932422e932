"""smerf_sample_noalloc, the entry point for callers that cannot let the library allocate
device memory (hosts whose device memory is carved out at start-up, frameworks that own
every device byte through their own pool).  Its output must equal smerf_sample's on the same plan and
seeds, call after call, since both run the same kernels; only the scratch location
differs (a fixed 16 MiB device array instead of the stream-ordered allocator).

Named test_zz_* so that pytest collects it last."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flags_name", ["fp32", "fp64", "fp64_tables"])
def test_noalloc_matches_allocating_entry_twice(flags_name):
    """Bit for bit: the same kernels on the same noise.  With FP64 tables and FP32 recursion
    and n >= 4, smerf_sample stages the tables as FP32 in its scratch while
    smerf_sample_noalloc converts them inside its kernels; both use the same truncating
    conversion, so the fields must still be identical."""
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_TABLES_FP64, Plan
    flags = {"fp32": 0, "fp64": SMERF_RECUR_FP64, "fp64_tables": SMERF_TABLES_FP64}[flags_name]
    kappa = [20.0, 50.0] if flags_name == "fp64_tables" else [10.0]
    plan = Plan(kappa, 1.0, 32, 64, flags=flags, anchor_spacing=8)
    for seed, n in [(3, 5), (11, 4)]:  # two calls in a row reuse the same fixed scratch
        ref = plan.sample(seed, n)
        got = torch.full_like(ref, float("nan"))
        plan.sample_noalloc(seed, n, got)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(got).all())
        assert torch.equal(got, ref)


def test_noalloc_p2_grid_and_rejects_oversize():
    import torch
    from paper_1709_10314_gb300 import Plan, SmerfError
    plan = Plan([20.0, 50.0], 1.0, 64, 128, anchor_spacing=8)
    ref = plan.sample(7, 4)
    got = torch.empty_like(ref)
    plan.sample_noalloc(7, 4, got)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    per = plan.info()["scratch_bytes_per_sample"]
    n_big = (16 << 20) // per + 1
    with pytest.raises(SmerfError) as e:
        plan.sample_noalloc(1, n_big, torch.empty((n_big, 64, 128), dtype=torch.float32, device="cuda"))
    assert e.value.status == -6
