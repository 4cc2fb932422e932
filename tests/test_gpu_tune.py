"""Launch-configuration autotuning: every candidate configuration of the segment kernel
(units per producer thread, realisations per CTA, producer and FFT threads, CTAs per SM the
kernel is built for, FFT radix plan) with the same radix plan produces the same field bit for
bit, the built-in choice among them; the two radix plans agree to FP32 rounding; the autotuner
picks one of the candidates, a fixed choice can be set and cleared, and a batch mixing a tuned
and an untuned plan of one shape is still exact."""
import pytest

pytestmark = pytest.mark.gpu


def _plan(flags=0, kappa=(20.0, 50.0), n_theta=48, n_phi=512, H=16):
    from paper_1709_10314_gb300 import Plan
    return Plan(list(kappa), 1.0, n_theta, n_phi, flags=flags, anchor_spacing=H)


@pytest.mark.parametrize("flags_name", ["fp32", "fp32_tables32", "fp64"])
def test_every_candidate_gives_the_same_field(flags_name):
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, SMERF_TABLES_FP32
    flags = {"fp32": 0, "fp32_tables32": SMERF_TABLES_FP32, "fp64": SMERF_RECUR_FP64}[flags_name]
    for kappa, n_phi, H in (((20.0, 50.0), 512, 16), ((30.0,), 1024, 8), ((10.0,), 64, 0)):
        plan = _plan(flags, kappa, 40, n_phi, H)
        cands = plan.launch_candidates()
        assert len(cands) >= 1
        ref = plan.sample(7, 5)   # 5 realisations: a ragged last group for 2 and 4 per CTA
        torch.cuda.synchronize()
        by_radix = {}
        for cfg in cands:
            upt, rmax, n_prod, n_fft, per_sm, radix = cfg
            assert n_prod % 32 == 0 and n_fft % 32 == 0 and n_prod + n_fft <= (768 if per_sm == 1 else 512)
            assert radix in (16, 4) and (radix == 4 or flags_name != "fp64")
            plan.set_launch(cfg)
            got = plan.sample(7, 5)
            torch.cuda.synchronize()
            first = by_radix.setdefault(radix, got)
            assert torch.equal(got, first), (flags_name, kappa, n_phi, cfg)
        # the built-in choice: the high-radix plan where there is one (FP32), else radix 4
        assert torch.equal(ref, by_radix[16] if 16 in by_radix else by_radix[4])
        if len(by_radix) == 2:
            d = (by_radix[16].double() - by_radix[4].double()).abs().max() / ref.double().std()
            assert float(d) < 1e-5, float(d)
        plan.set_launch(None)
        assert torch.equal(plan.sample(7, 5), ref)


def test_autotune_picks_a_candidate():
    import torch
    plan = _plan()
    ref = plan.sample(3, 4)
    chosen = plan.autotune(8)
    assert chosen in plan.launch_candidates()
    got = plan.sample(3, 4)
    torch.cuda.synchronize()
    if chosen[5] == 16:   # the built-in radix plan: the same field bit for bit
        assert torch.equal(got, ref)
    else:
        assert float((got.double() - ref.double()).abs().max() / ref.double().std()) < 1e-5


def test_set_launch_rejects_non_candidates():
    from paper_1709_10314_gb300 import SmerfError
    plan = _plan()
    with pytest.raises(SmerfError):
        plan.set_launch((3, 1, 96, 64, 1, 16))
    with pytest.raises(SmerfError):
        plan.set_launch((1, 4, 32, 800, 1, 16))
    with pytest.raises(SmerfError):
        plan.set_launch((2, 4, 512, 128, 2, 16))   # not built for two CTAs per SM
    with pytest.raises(SmerfError):
        plan.set_launch((2, 4, 256, 128, 1, 8))    # no radix-8 plan
    with pytest.raises(ValueError):
        plan.set_launch((2, 4, 256, 128, 1))       # six integers


def test_batch_with_tuned_and_untuned_plans_of_one_shape():
    import torch
    from paper_1709_10314_gb300 import Batch
    a, b = _plan(kappa=(20.0, 50.0)), _plan(kappa=(15.0, 45.0))
    cands = a.launch_candidates()
    pick = [c for c in cands if c[1] != cands[0][1]] or cands
    a.set_launch(pick[-1])
    counts = [3, 5]
    bt = Batch([a, b], counts)
    assert bt.info()["groups"] == 2   # the tuned plan forms its own group
    outs = [torch.empty((n, p.n_theta, p.n_phi), dtype=p.dtype, device="cuda") for p, n in zip([a, b], counts)]
    bt.sample([5, 6], outs)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], a.sample(5, 3))
    assert torch.equal(outs[1], b.sample(6, 5))


def test_autotune_anchor_spacing():
    """smerf_plan_autotune_anchor rebuilds the tables for each candidate spacing, keeps the
    fastest, and the tuned plan then samples exactly what a plan made with that spacing does."""
    import torch
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, Plan
    plan = Plan([20.0, 50.0], 1.0, 128, 256, anchor_spacing=16)
    h = plan.autotune_anchor(4, candidates=(8, 16, 32))
    assert h in (8, 16, 32) and plan.info()["anchor_spacing"] == h
    ref = Plan([20.0, 50.0], 1.0, 128, 256, anchor_spacing=h).sample(9, 4)
    got = plan.sample(9, 4)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    paper = Plan([20.0, 50.0], 1.0, 64, 128, flags=SMERF_ORDER_PAPER)
    assert paper.autotune_anchor(2, candidates=(8,)) == 0  # Alg. 2's order has no anchors
