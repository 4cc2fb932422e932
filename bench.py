#!/usr/bin/env python
"""Throughput of the GB300 sphere-GMRF sampler on its headline workload.

Workload (default): 1024 x 2048 equiangular grid, C_l = 1/((l(l+1)+20^2)(l(l+1)+50^2))
(p = 2), 64 realisations per step, FP64 tables, FP32 recursion + FFT, anchors every 16
rings.  A step is one smerf_sample call: the anchor kernel and the segment kernel that
synthesises and writes every ring.  Metric: sphere grid points per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  --impl reference times the oracle (the FP64 CPU
restatement of the method) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KAPPA = [20.0, 50.0]
AMP = 1.0
N_THETA, N_PHI, N_REAL, ANCHOR, SEED = 1024, 2048, 64, 16, 1
WORKLOAD = ("1024x2048 equiangular grid, C_l=1/((l(l+1)+20^2)(l(l+1)+50^2)) (p=2), 64 realisations, "
            "FP64 tables, FP32 recursion+FFT")
METRIC = "sphere grid points/s"
FLUSH_BYTES = 256 << 20


SMS, FP32_LANES, FP64_PER_SM = 152, 128, 2     # GB300: SMs, FP32 lanes per SM, FP64 FMAs per SM per clock


def alg_ops_per_item(p, Nc, fp64=False):
    """Algorithmic ALU operations of one (mode, realisation, ring) item of the method (an FMA
    counts as one): Philox4x32-10 (10 rounds x 2 widening multiplies + 2 three-input XORs per
    call of 4 normals), Box-Muller (12 per pair: 2 conversions, 2 scalings, log2, scaling,
    rsqrt, product, sin, cos, 2 products), the recursion x = A x + B xi on the Re and Im
    chains (Eq. (state_space)), and this item's share of the ring's C2R FFT (10 for the
    packing, 3.5 log2 Nc for a radix-4 complex FFT).  With fp64 only the floating-point part
    (Box-Muller, recursion, FFT), which runs on the FP64 pipe."""
    philox = 40.0 * (2 * p) / 4.0
    box_muller = 12.0 * p
    recursion = 2.0 * (p * p + p * (p + 1) / 2.0)
    fft = 10.0 + 3.5 * math.log2(Nc)
    return (box_muller + recursion + fft) if fp64 else (philox + box_muller + recursion + fft)


def alu_peak(fp64, sm_mhz):
    """Lane operations per second: FP32 (and INT32) issue 128 lanes per SM per clock; FP64 2."""
    return SMS * (FP64_PER_SM if fp64 else FP32_LANES) * sm_mhz * 1e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler for the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def csrc_digest():
    """Digest of the sources the sampling kernels are built from (their templates and their
    instantiation units); the committed DRAM-traffic record is valid while it matches."""
    import glob
    import hashlib
    h = hashlib.sha256()
    base = os.path.join(ROOT, "paper_1709_10314_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(base, "smerf_sample_*.cu")) +
                    [os.path.join(base, "smerf_sample_impl.cuh"), os.path.join(base, "smerf_internal.cuh")]):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def oracle_sample_step(n_real=1, seed=SEED):
    """The oracle on a bounded sample of the workload: the start ring (k0) of n_real
    realisations, including the oracle's own covariance construction for that ring."""
    import oracle
    order = oracle.conditioning_order(N_THETA, ANCHOR)
    t0 = time.perf_counter()
    oracle.sample(KAPPA, AMP, N_THETA, N_PHI, seed, n_real, H=ANCHOR, rings=order[:1])
    return time.perf_counter() - t0, n_real * N_PHI


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return
    dts = []
    for i in range(args.warmup + args.steps):
        dt, pts = oracle_sample_step()
        if i >= args.warmup:
            dts.append(dt)
    ms = 1e3 * sum(dts) / len(dts)
    value = pts / (ms / 1e3)
    sample = "start ring (k0=512) of 1 realisation of the workload per step (2048 points), oracle incl. its covariance sums"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if (args.tables or "fp64") == "fp64" else WORKLOAD.replace("FP64 tables", "FP32 tables"),
                       "n_theta": N_THETA, "n_phi": N_PHI},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gb300(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1709_10314_gb300 import Batch, Plan, create_plans
    from paper_1709_10314_gb300.replicas import max_over_ranks, rank_seed
    from paper_1709_10314_gb300.workloads import FIXED, TUNED_LAUNCH, flags_for, uneven_requests

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = args.workload
    batch = None
    launch_cfg = None
    if wl == "uneven-256":
        reqs = uneven_requests()
        # all 256 plans made in one call, their set-ups overlapping on the GPU
        plans = create_plans([dict(kappa=r["kappa"], A=r["A"], n_theta=r["n_theta"], n_phi=r["n_phi"],
                                   flags=flags_for("fp32", args.tables or "fp32")) for r in reqs])
        counts = [r["n"] for r in reqs]
        base_seeds = [r["seed"] for r in reqs]
        # with --tune: launch configurations tuned once per request shape (set-up, untimed; by
        # default the built-in choice, which measured faster for the whole batch)
        if args.tune:
            shapes = {}
            for p_, n_ in zip(plans, counts):
                key = (p_.info()["p"], p_.n_theta, p_.n_phi)
                shapes.setdefault(key, []).append((p_, n_))
            for key, members in shapes.items():
                rep = max(members, key=lambda t: t[1])
                if rep[0].launch_candidates():
                    best = rep[0].autotune(rep[1])
                    for p_, _ in members:
                        p_.set_launch(best)
        outs = [torch.empty((n, p.n_theta, p.n_phi), dtype=torch.float32, device=dev) for p, n in zip(plans, counts)]
        batch = Batch(plans, counts)
        points = sum(n * p.n_theta * p.n_phi for p, n in zip(plans, counts))
        fp64_alu = False
        alg_ops = sum(n * p.n_theta * (p.n_phi // 2) * alg_ops_per_item(p.info()["p"], p.n_phi // 2)
                      for p, n in zip(plans, counts))
        table_bytes = sum(p.info()["table_bytes"] for p in plans)
        out_bytes = points * 4
        workload = ("uneven batch: 256 requests, n_theta in {128,256,512,1024}, n_phi=2 n_theta, kappa in [5,200], "
                    "p in {1,2}, 1-8 realisations, FP32 recursion, FP%s tables, one CUDA-graph replay per step"
                    % ("64" if args.tables == "fp64" else "32"))
        dtype = "f32"
        setup_ms = plans[0].info()["setup_ms"]  # the wall time of the one call that made them all
        s_cap = torch.cuda.Stream(device=dev)

        def set_seeds(step):
            off = rank_seed(0, rank, 1 << 40) + (step << 20)
            batch.set([b_ + off for b_ in base_seeds], outs)

        set_seeds(0)
        with torch.cuda.stream(s_cap):
            batch.launch(stream=s_cap)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s_cap, capture_error_mode="relaxed"):
            batch.launch(stream=s_cap)
        launches = 2 * batch.info()["groups"] + batch.info()["singles"] * 2

        def step(i, ev0=None, ev1=None):
            torch.cuda.synchronize()
            set_seeds(i)
            if ev0 is not None:
                ev0.record()
            graph.replay()
            if ev1 is not None:
                ev1.record()
    else:
        cfg = dict(FIXED[wl])
        recur = args.recur or cfg["recur"]
        tables = args.tables or cfg["tables"]
        from paper_1709_10314_gb300 import SMERF_ORDER_PAPER
        paper_order = cfg.get("order") == "paper"
        plan = Plan(cfg["kappa"], cfg["A"], cfg["n_theta"], cfg["n_phi"],
                    flags=flags_for(recur, tables) | (SMERF_ORDER_PAPER if paper_order else 0),
                    anchor_spacing=0 if paper_order else ANCHOR)
        info = plan.info()
        n = cfg["n"]
        # launch configuration of the segment kernel: timed candidates (set-up, untimed)
        ws_kernel = len(plan.launch_candidates()) > 0
        stored = TUNED_LAUNCH.get((wl, recur, tables))
        if args.launch and ws_kernel:
            launch_cfg = [int(v) for v in args.launch.split(",")]
            plan.set_launch(launch_cfg)
        elif ws_kernel and not args.no_tune and not args.tune and stored in plan.launch_candidates():
            launch_cfg = list(stored)
            plan.set_launch(launch_cfg)
        else:
            launch_cfg = list(plan.autotune(n)) if (ws_kernel and not args.no_tune) else None
        out = torch.empty((n, cfg["n_theta"], cfg["n_phi"]), dtype=plan.dtype, device=dev)
        points = n * cfg["n_theta"] * cfg["n_phi"]
        out_bytes = points * (8 if recur == "fp64" else 4)
        fp64_alu = recur == "fp64"
        alg_ops = n * cfg["n_theta"] * (cfg["n_phi"] // 2) * alg_ops_per_item(len(cfg["kappa"]), cfg["n_phi"] // 2, fp64_alu)
        table_bytes = info["table_bytes"]
        # what the segment kernel reads: the step tables and the anchor states
        seg_read_bytes = info["step_table_bytes"], n * info["scratch_bytes_per_sample"]
        setup_ms = info["setup_ms"]
        dtype = "f64" if recur == "fp64" else "f32"
        workload = "%dx%d equiangular grid, C_l=1/prod(l(l+1)+kappa^2) kappa=%s (p=%d), %d realisations, %s tables, %s recursion+FFT" % (
            cfg["n_theta"], cfg["n_phi"], "(" + ",".join("%g" % k for k in cfg["kappa"]) + ")", len(cfg["kappa"]), n,
            tables.upper(), recur.upper())
        launches = plan.launches(n)
        seed0 = rank_seed(cfg["seed"], rank, n * (args.warmup + args.steps + 8))

        def step(i, ev0=None, ev1=None):
            if ev0 is not None:
                ev0.record()
            plan.sample_timed(seed0 + i * n, n, out, s0[i], s1[i]) if ev0 is not None else plan.sample(seed0 + i * n, n, out)
            if ev1 is not None:
                ev1.record()

    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0 = [ev() for _ in range(args.steps)]
    e1 = [ev() for _ in range(args.steps)]
    s0 = [ev() for _ in range(args.steps)]
    s1 = [ev() for _ in range(args.steps)]
    # the clock sampler starts first, so that the warm-up steps (not an idle pause) directly
    # precede the timed ones
    clk = Clocks(local_rank)
    clk.start()
    time.sleep(0.3)
    for w in range(args.warmup):
        step(args.steps + w)
        flush.fill_(float(w))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    for i in range(args.steps):
        step(i, e0[i], e1[i])
        flush.fill_(float(i))  # L2 flush between timed steps (outside the step events)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / args.steps
    if batch is None:
        seg_ms = sum(a.elapsed_time(b) for a, b in zip(s0, s1)) / args.steps
        kernel = "segment_ws_kernel" if ws_kernel else "segment_kernel"
    else:
        seg_ms = step_ms  # the graph replay: all groups' anchor + segment launches
        kernel = "batched graph replay (anchor + segment launches of every group)"
    step_ms, seg_ms = max_over_ranks([step_ms, seg_ms], device=dev)
    value = world * points / (step_ms / 1e3)

    # Rooflines of the segment kernel.  It is bound by ALU issue (noise, recursion and FFT
    # arithmetic), not by HBM: ALU = algorithmic operations / kernel time against the lane
    # rate at the maximum SM clock; HBM = field written once + step tables and anchor states
    # read once.  (FP64 tables with FP32 recursion: each call stages the step tables as FP32
    # once; the segment kernel reads that copy, half their bytes.)  The batched graph replay
    # (anchor and segment launches) counts the field and all of its plans' tables.
    staged = batch is None and (args.recur or FIXED[wl]["recur"]) == "fp32" and \
        (args.tables or FIXED[wl]["tables"]) == "fp64" and FIXED[wl]["n"] >= 4
    if batch is None:
        step_b, anc_b = seg_read_bytes
        alg_bytes = out_bytes + (step_b // 2 if staged else step_b) + anc_b
    else:
        alg_bytes = out_bytes + table_bytes
    peak, peak_kind = _peaks()
    achieved = alg_bytes / (seg_ms / 1e3) / 1e9
    sm_max = float(clocks.get("sm_max_mhz") or 2070.0) if isinstance(clocks, dict) else 2070.0
    alu_pk = alu_peak(fp64_alu, sm_max) / 1e9
    alu_ach = alg_ops / (seg_ms / 1e3) / 1e9
    # DRAM traffic of one segment-kernel launch from the committed ncu record, only while the
    # kernel sources still hash to what was profiled (null otherwise)
    traffic = None
    prof = os.path.join(ROOT, "profiles", "segment_kernel_traffic.json")
    if os.path.exists(prof) and not args.recur and args.tables is None and batch is None:
        try:
            rec = json.load(open(prof))
            w = rec.get("workloads", {}).get(wl)
            if w and rec.get("csrc_sha256_16") == csrc_digest() and w.get("launch") == launch_cfg:
                traffic = w.get("traffic_bytes_per_launch")
        except Exception:
            traffic = None

    # end to end through the C ABI with host buffers (the field crosses the CPU-GPU link inside
    # the timed region): smerf_sample_host, or the batch writing page-locked host outputs
    e2e = None
    if batch is not None:
        host_outs = [torch.empty(tuple(o.shape), dtype=o.dtype, pin_memory=True) for o in outs]
        off = rank_seed(0, rank, 1 << 40) + ((args.steps + args.warmup + 1) << 20)
        batch.sample([b_ + off for b_ in base_seeds], host_outs)
        torch.cuda.synchronize()
        ne = 3
        t0 = time.perf_counter()
        for i in range(ne):
            batch.sample([b_ + off + ((i + 1) << 20) for b_ in base_seeds], host_outs)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / ne
        e2e = {"value": world * points / e2e_s, "unit": "points/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": out_bytes}
    else:
        host = torch.empty(tuple(out.shape), dtype=out.dtype, pin_memory=True)
        plan.sample_host(seed0, n, host)
        ne = 3
        t0 = time.perf_counter()
        for i in range(ne):
            plan.sample_host(seed0 + i * n, n, host)
        e2e_s = (time.perf_counter() - t0) / ne
        e2e = {"value": world * points / e2e_s, "unit": "points/s", "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": out_bytes}

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline and wl == "1024x2048-p2":
        dt, pts = oracle_sample_step(n_real=4)
        cpu = {"value": pts / dt, "unit": "points/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "start ring (k0=512) of realisations 1-4 of the workload (4 x 2048 points), "
                         "the oracle's spectral-sum covariance, Cholesky, Philox noise and naive DFT"}
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": workload, "name": wl, "points_per_gpu": points, "anchor_spacing": ANCHOR,
                       "launch": launch_cfg, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between timed steps (256 MiB write outside the step events)"},
            "roofline": {"bound": "alu", "achieved": alu_ach, "peak": alu_pk, "unit": "Gop/s",
                         "frac": alu_ach / alu_pk, "traffic": traffic,
                         "peak_kind": "derived: %d SMs x %d %s lanes x %.0f MHz" % (
                             SMS, FP64_PER_SM if fp64_alu else FP32_LANES, "FP64" if fp64_alu else "FP32/INT32", sm_max),
                         "algorithmic_ops": alg_ops, "kernel": kernel, "kernel_ms": seg_ms,
                         "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                 "peak_kind": peak_kind, "algorithmic_bytes": alg_bytes,
                                 "tables_staged_fp32": staged}},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches * args.steps,
            "clocks": clocks,
            "setup_ms": setup_ms, "table_bytes": table_bytes}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tables", default=None, choices=["fp64", "fp32"],
                    help="override the workload's table storage precision")
    ap.add_argument("--recur", default=None, choices=["fp64", "fp32"],
                    help="override the workload's recursion precision")
    ap.add_argument("--tune", action="store_true",
                    help="time the launch candidates (smerf_plan_autotune) instead of the stored choice")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the built-in segment-kernel launch configuration (no autotuning)")
    ap.add_argument("--launch", default=None,
                    help="fix the segment-kernel launch configuration: units/thread,realisations/CTA,"
                         "producer threads,FFT threads (one of the plan's candidates)")
    ap.add_argument("--workload", default="1024x2048-p2",
                    choices=["1024x2048-p2", "plain-64x128-p1-fp64", "4096x8192-p1", "16384x32768-p1", "uneven-256"])
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_gb300(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
