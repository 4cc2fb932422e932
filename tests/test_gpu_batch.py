"""Batched sampling: requests of different grids, spectra, p and precision in grouped
launches (one anchor and one segment launch per kernel shape) give exactly what
individual smerf_sample calls give; a batch is reusable and replays under a CUDA graph
with new seeds."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _plans():
    from paper_1709_10314_gb300 import SMERF_ORDER_PAPER, SMERF_RECUR_FP64, SMERF_TABLES_FP64, Plan
    specs = [
        ([10.0], 32, 64, 0, 8),
        ([20.0, 50.0], 64, 128, 0, 16),
        ([5.0], 17, 64, 0, 4),                    # same shape as the first: one group
        ([3.0, 8.0], 24, 32, SMERF_RECUR_FP64, 4),
        ([7.0], 40, 256, SMERF_TABLES_FP64, 0),
        ([9.0, 30.0], 16, 32, SMERF_ORDER_PAPER, 0),
    ]
    return [Plan(k, 1.0, nt, nphi, flags=f, anchor_spacing=H) for (k, nt, nphi, f, H) in specs]


def _outs(plans, counts):
    import torch
    return [torch.full((n, p.n_theta, p.n_phi), float("nan"), dtype=p.dtype, device="cuda")
            for p, n in zip(plans, counts)]


def test_batched_equals_single_calls():
    import torch
    from paper_1709_10314_gb300 import sample_batched
    plans = _plans()
    counts = [3, 5, 1, 2, 6, 2]
    seeds = [11, 22, 33, 44, 55, 66]
    outs = _outs(plans, counts)
    sample_batched(plans, seeds, counts, outs)
    torch.cuda.synchronize()
    for p, s, n, o in zip(plans, seeds, counts, outs):
        ref = p.sample(s, n)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


def test_batch_object_reuse_and_groups():
    import torch
    from paper_1709_10314_gb300 import Batch
    plans = _plans()
    counts = [2, 2, 2, 1, 3, 1]
    b = Batch(plans, counts)
    info = b.info()
    assert info["groups"] == 5 and info["singles"] == 0   # plans 0 and 2 share a shape
    # FP32 recursion with FP32 tables (plans 0, 1, 2, 5) and with FP64 tables (plan 4): an anchor
    # launch and a persistent launch each (one persistent launch each in the single-launch
    # form); FP64 recursion (plan 3): an anchor and a segment launch
    assert info["launches"] == 6
    b.set_single_launch(True)
    assert b.info()["launches"] == 4
    for single, seeds in ((False, [1, 2, 3, 4, 5, 6]), (True, [100, 200, 300, 400, 500, 600])):
        b.set_single_launch(single)
        outs = _outs(plans, counts)
        b.sample(seeds, outs)
        assert b.status() == 0
        torch.cuda.synchronize()
        for p, s, n, o in zip(plans, seeds, counts, outs):
            assert torch.equal(o, p.sample(s, n))


@pytest.mark.parametrize("single", [False, True])
def test_batch_cuda_graph_replay(single):
    import torch
    from paper_1709_10314_gb300 import Batch
    plans = _plans()[:3]
    counts = [4, 2, 3]
    b = Batch(plans, counts)
    b.set_single_launch(single)
    outs = _outs(plans, counts)
    b.set([1, 2, 3], outs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.launch(stream=s)   # first launch outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        b.launch(stream=s)
    for seeds in ([7, 8, 9], [70, 80, 90]):
        torch.cuda.synchronize()
        b.set(seeds, outs)
        g.replay()
        torch.cuda.synchronize()
        assert b.status() == 0
        for p, sd, n, o in zip(plans, seeds, counts, outs):
            assert torch.equal(o, p.sample(sd, n))


def test_batch_writes_pinned_host_outputs():
    # page-locked host outputs: the kernels write them over the CPU-GPU link; the same fields
    import torch
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, Batch, Plan
    plans = [Plan([10.0], 1.0, 32, 64, anchor_spacing=8), Plan([3.0, 8.0], 1.0, 17, 32, anchor_spacing=4),
             Plan([4.0], 1.0, 16, 32, flags=SMERF_RECUR_FP64, anchor_spacing=4)]
    counts = [3, 2, 2]
    b = Batch(plans, counts)
    dev = [torch.empty((n, p.n_theta, p.n_phi), dtype=p.dtype, device="cuda") for p, n in zip(plans, counts)]
    host = [torch.full((n, p.n_theta, p.n_phi), float("nan"), dtype=p.dtype, pin_memory=True)
            for p, n in zip(plans, counts)]
    b.sample([5, 6, 7], dev)
    torch.cuda.synchronize()
    b.sample([5, 6, 7], host)
    torch.cuda.synchronize()
    for d, h in zip(dev, host):
        assert torch.equal(d.cpu(), h)


def test_batch_graph_replay_against_oracle():
    """A graph-replayed batch checked against the oracle directly, not only against single
    calls: three requests of different shapes (two FP32 grids, one FP64 with p = 2), each
    replay with new seeds; every ring of every realisation within the parity tolerances
    (FP32 1e-4, FP64 1e-9 of the field std)."""
    import torch
    import oracle
    from paper_1709_10314_gb300 import SMERF_RECUR_FP64, Batch, Plan
    specs = [([10.0], 32, 64, 0, 8, 3), ([5.0], 17, 64, 0, 8, 2), ([3.0, 8.0], 24, 32, SMERF_RECUR_FP64, 4, 2)]
    plans = [Plan(k, 1.0, nt, nphi, flags=f, anchor_spacing=H) for (k, nt, nphi, f, H, _) in specs]
    counts = [s[-1] for s in specs]
    b = Batch(plans, counts)
    outs = _outs(plans, counts)
    b.set([1, 2, 3], outs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.launch(stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        b.launch(stream=s)
    for seeds in ([7, 8, 9], [1000, 2000, 3000]):
        torch.cuda.synchronize()
        b.set(seeds, outs)
        g.replay()
        torch.cuda.synchronize()
        for (k, nt, nphi, f, H, n), sd, o in zip(specs, seeds, outs):
            ref = oracle.sample(k, 1.0, nt, nphi, sd, n, H=H)
            err = float(np.max(np.abs(o.double().cpu().numpy() - ref))) / float(np.std(ref))
            assert err < (1e-9 if f else 1e-4), (k, nt, nphi, sd, err)


@pytest.mark.parametrize("single", [False, True])
def test_uneven_batch_persistent_launches(single):
    """Requests of four grids and both p with FP32 recursion: an anchor launch and one launch of
    persistent CTAs that pull every shape's segments from the device queue, or (single) one
    launch of persistent CTAs that pull every request's anchor items and then every segment;
    each request bit for bit what its own smerf_sample call gives, launch after launch."""
    import torch
    from paper_1709_10314_gb300 import Batch, Plan
    specs = [([12.0], 128, 256, 3), ([30.0, 90.0], 256, 512, 2), ([7.0], 64, 128, 5), ([20.0, 50.0], 512, 1024, 1),
             ([150.0], 1024, 2048, 2), ([40.0, 130.0], 128, 256, 4)]
    plans = [Plan(k, 1.0, nt, nphi) for (k, nt, nphi, _) in specs]
    counts = [s[-1] for s in specs]
    b = Batch(plans, counts)
    b.set_single_launch(single)
    assert b.info()["launches"] == (1 if single else 2) and b.info()["singles"] == 0
    for rep in range(3):
        seeds = [5 * i + 1 + 1000 * rep for i in range(len(plans))]
        outs = _outs(plans, counts)
        b.sample(seeds, outs)
        assert b.status() == 0
        for p, sd, n, o in zip(plans, seeds, counts, outs):
            assert torch.equal(o, p.sample(sd, n))


def test_anchor_wait_that_runs_out_is_reported_and_the_batch_recovers():
    """The persistent launch's one device wait (a segment item waiting for its request's anchor
    items) is bounded: with the anchor counters started one below zero (the test hook) no wait
    can be met, the first runs out after about a second, the others give up at once, and
    smerf_batch_status reports SMERF_ETIMEOUT with the context still usable.  The next launch
    is normal and exact."""
    import time
    import torch
    from paper_1709_10314_gb300 import Batch, Plan
    plans = [Plan([12.0], 1.0, 64, 128), Plan([30.0, 90.0], 1.0, 128, 256)]
    counts = [2, 3]
    b = Batch(plans, counts)
    b.set_single_launch(True)
    outs = _outs(plans, counts)
    for o in outs:
        o.fill_(float("nan"))
    b.debug_fail_waits()
    t0 = time.perf_counter()
    b.sample([1, 2], outs)
    assert b.status() == -7
    assert time.perf_counter() - t0 < 30.0
    assert all(bool(torch.isnan(o).all()) for o in outs)   # no segment ran: no ring written
    b.sample([1, 2], outs)
    assert b.status() == 0
    for p, sd, n, o in zip(plans, [1, 2], counts, outs):
        assert torch.equal(o, p.sample(sd, n))
