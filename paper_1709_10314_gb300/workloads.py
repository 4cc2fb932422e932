"""Synthetic workloads (inputs only: grids, spectra, realisation counts and seeds; no part
of the method's arithmetic).  Each is named by what it is.

  plain-64x128-p1-fp64      64 x 128, C_l = 1/(l(l+1)+10^2), 1 realisation, FP64 recursion
  1024x2048-p2              1024 x 2048, C_l = 1/((l(l+1)+20^2)(l(l+1)+50^2)), 64 realisations,
                            FP64 tables, FP32 recursion + FFT (the throughput workload)
  1024x2048-p3              1024 x 2048, C_l = 1/((l(l+1)+20^2)(l(l+1)+50^2)(l(l+1)+120^2)),
                            64 realisations, FP64 tables, FP32 recursion + FFT (three factors)
  4096x8192-p1              4096 x 8192, C_l = 1/(l(l+1)+100^2), 16 realisations (precision sweep:
                            recursion FP64/FP32 x tables FP64/FP32)
  uneven-256                256 requests: n_theta uniform in {128,256,512,1024}, n_phi = 2 n_theta,
                            kappa uniform in [5, 200], p uniform in {1, 2}, 1-8 realisations,
                            FP32 recursion; generator seed 12345, request i draws keys 1000 i + j
  16384x32768-p1            16384 x 32768, C_l = 1/(l(l+1)+300^2), 4 realisations, FP32 tables,
                            anchors every 24 rings (measured best of 16, 24, 32)
  4096x32768-p1             the same spectrum, ring length and realisations on a quarter of the
                            rings (4096): the same kernels at a size for profiling captures
"""
import numpy as np

FIXED = {
    "plain-64x128-p1-fp64": dict(kappa=[10.0], A=1.0, n_theta=64, n_phi=128, n=1, seed=1,
                                 recur="fp64", tables="fp64", order="paper"),
    "1024x2048-p2": dict(kappa=[20.0, 50.0], A=1.0, n_theta=1024, n_phi=2048, n=64, seed=1,
                         recur="fp32", tables="fp64"),
    "1024x2048-p3": dict(kappa=[20.0, 50.0, 120.0], A=1.0, n_theta=1024, n_phi=2048, n=64, seed=1,
                         recur="fp32", tables="fp64"),
    "4096x8192-p1": dict(kappa=[100.0], A=1.0, n_theta=4096, n_phi=8192, n=16, seed=1,
                         recur="fp32", tables="fp64"),
    "16384x32768-p1": dict(kappa=[300.0], A=1.0, n_theta=16384, n_phi=32768, n=4, seed=1,
                           recur="fp32", tables="fp32", H=24),
    "4096x32768-p1": dict(kappa=[300.0], A=1.0, n_theta=4096, n_phi=32768, n=4, seed=1,
                          recur="fp32", tables="fp32", H=24),
}

# Segment-kernel launch configurations (units per producer thread, realisations per CTA,
# producer threads, FFT threads, CTAs per SM, FFT radix plan) that smerf_plan_autotune chose on
# a GB300, per (workload, recursion precision, table precision); bench.py uses them unless asked
# to re-tune.
TUNED_LAUNCH = {
    ("1024x2048-p2", "fp32", "fp64"): (4, 1, 256, 64, 2, 16),
    ("1024x2048-p2", "fp32", "fp32"): (4, 1, 256, 64, 2, 16),
    ("1024x2048-p2", "fp64", "fp64"): (4, 1, 256, 128, 1, 4),
    ("1024x2048-p3", "fp32", "fp64"): (4, 1, 128, 32, 1, 16),
    ("4096x8192-p1", "fp32", "fp64"): (4, 1, 512, 256, 1, 16),
    ("plain-64x128-p1-fp64", "fp64", "fp64"): (1, 1, 32, 32, 1, 4),
}


def uneven_requests(n_req=256, gen_seed=12345):
    """The uneven batch: list of dicts (kappa, n_theta, n_phi, n, seed).  kappa pairs whose
    squares are within 1e-3 relative are redrawn (partial fractions would cancel)."""
    rng = np.random.default_rng(gen_seed)
    reqs = []
    for i in range(n_req):
        n_theta = int(rng.choice([128, 256, 512, 1024]))
        p = int(rng.integers(1, 3))
        while True:
            kappa = sorted(float(v) for v in rng.uniform(5.0, 200.0, size=p))
            if p == 1 or abs(kappa[0] ** 2 - kappa[1] ** 2) > 1e-3 * kappa[1] ** 2:
                break
        reqs.append(dict(kappa=kappa, A=1.0, n_theta=n_theta, n_phi=2 * n_theta,
                         n=int(rng.integers(1, 9)), seed=1000 * i))
    return reqs


def flags_for(recur, tables):
    from .smerf import SMERF_RECUR_FP64, SMERF_TABLES_FP32, SMERF_TABLES_FP64
    f = SMERF_RECUR_FP64 if recur == "fp64" else 0
    f |= SMERF_TABLES_FP64 if tables == "fp64" else SMERF_TABLES_FP32
    return f
