"""GB300-native sampler for isotropic Gaussian Markov random fields on the sphere
(Creasey & Lang, "Fast generation of isotropic Gaussian random fields on the sphere",
arXiv 1709.10314).

Every step of the sampling path runs in the CUDA library ``libsmerf.so`` (C ABI in
``include/smerf.h``); this package only marshals arguments.  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing the binding fails loudly when
the library has not been built (``python -m paper_1709_10314_gb300.build``).
"""
from .smerf import (  # noqa: F401
    SMERF_ORDER_PAPER, SMERF_RECUR_FP64, SMERF_TABLES_FP32, SMERF_TABLES_FP64, Batch, Plan, SmerfError,
    create_plans, debug_fail_alloc, last_device_status, library_path, philox_uint32, ring_normals, sample_batched,
    scratch_trim,
)
