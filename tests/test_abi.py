"""The C ABI library loads and exports every entry point include/smerf.h declares;
argument validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smerf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1709_10314_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(smerf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["smerf_plan_create", "smerf_plan_create_ex", "smerf_sample", "smerf_sample_batched",
              "smerf_plan_destroy", "smerf_sample_host", "smerf_plan_info"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def _create(lib, kappa, p, A, nt, nphi, flags=0, H=0):
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    h = ctypes.c_void_p()
    lib.smerf_plan_create_ex.restype = ctypes.c_int
    rc = lib.smerf_plan_create_ex(k.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p, ctypes.c_double(A),
                                  nt, nphi, ctypes.c_uint(flags), H, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("args,code", [
    (([1.0], 0, 1.0, 16, 32), -1),              # p < 1
    (([-1.0], 1, 1.0, 16, 32), -1),             # kappa <= 0
    (([float("nan")], 1, 1.0, 16, 32), -1),     # non-finite kappa
    (([1.0], 1, 0.0, 16, 32), -1),              # A <= 0
    (([1.0], 1, 1.0, 1, 32), -1),               # n_theta < 2
    (([1.0], 1, 1.0, 16, 31), -1),              # odd n_phi
    (([3.0, 3.0000000001], 2, 1.0, 16, 32), -2),  # near-equal kappa: partial fractions cancel
    (([1.0], 1, 1.0, 16, 48), -5),              # n_phi not a power of two
    (([1.0, 2.0, 3.0, 4.0], 4, 1.0, 16, 32), -1),  # p > 3
    (([2.0, 5.0, 5.0000000001], 3, 1.0, 16, 32), -2),  # p = 3 with near-equal kappa
    (([2.0, 5.0, 9.0], 3, 1.0, 16, 16384), -5),  # p = 3 rings longer than 4096 complex points
])
def test_validation_without_gpu(lib, args, code):
    rc, h = _create(lib, *args)
    assert rc == code and not h.value


def test_bad_flags_and_spacing(lib):
    assert _create(lib, [1.0], 1, 1.0, 16, 32, flags=0x100)[0] == -1
    assert _create(lib, [1.0], 1, 1.0, 16, 32, flags=0x6)[0] == -1      # FP32 and FP64 tables
    assert _create(lib, [1.0], 1, 1.0, 16, 32, H=-3)[0] == -1


def test_launch_count_validation(lib):
    lib.smerf_sample_launches.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.smerf_sample_launches.restype = ctypes.c_int
    assert lib.smerf_sample_launches(None, 4) == -1


def test_status_strings(lib):
    lib.smerf_status_string.restype = ctypes.c_char_p
    assert lib.smerf_status_string(0) == b"ok"
    assert b"argument" in lib.smerf_status_string(-1)
    assert lib.smerf_plan_destroy(None) == 0


def test_khat_validation_without_gpu(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.smerf_plan_create_khat.restype = ctypes.c_int
    out = ctypes.c_void_p()

    def call(re, im, p):
        r = (ctypes.c_double * len(re))(*re)
        i = (ctypes.c_double * len(im))(*im)
        return lib.smerf_plan_create_khat(ctypes.cast(r, dp), ctypes.cast(i, dp), p, ctypes.c_double(1.0), 16, 32,
                                          0, 0, ctypes.byref(out))
    assert call([1.0, 1.0], [2.0, 3.0], 2) == -1      # not a conjugate pair
    assert call([1.0], [2.0], 1) == -1                # a single complex value
    assert call([1.0, 2.0], [2.0, -2.0], 2) == -1     # real parts differ
    assert call([1.0, 1.0], [1e-9, -1e-9], 2) == -2   # nearly a double root: ill-conditioned
    assert call([-1.0], [0.0], 1) == -1               # real kappa-hat must be > 0
    assert call([0.0, 0.0, -4.0], [3.0, -3.0, 0.0], 3) == -1   # p = 3: pair and a real value <= 0
    assert call([0.0, 0.0, 1.0], [3.0, -3.0, 2.0], 3) == -1    # p = 3: pair and an unpaired complex value
    assert call([5.0, 0.0, 0.0], [0.0, 3.0, 2.0], 3) == -1     # p = 3: real value, then no conjugate pair


def test_colatitude_validation_without_gpu(lib):
    """smerf_plan_create_theta rejects colatitudes that are not finite and strictly increasing
    inside (0, pi), and bad spectra, before it touches a GPU."""
    dp = ctypes.POINTER(ctypes.c_double)
    lib.smerf_plan_create_theta.restype = ctypes.c_int
    out = ctypes.c_void_p()
    n = 8
    good = [np.pi * (k + 0.5) / n for k in range(n)]

    def call(theta, kappa=(10.0,), nt=n):
        k = np.ascontiguousarray(kappa, dtype=np.float64)
        t = np.ascontiguousarray(theta, dtype=np.float64)
        return lib.smerf_plan_create_theta(k.ctypes.data_as(dp), len(kappa), ctypes.c_double(1.0), nt,
                                           t.ctypes.data_as(dp), 32, ctypes.c_uint(0), 0, ctypes.byref(out))
    assert call(good[::-1]) == -1                          # decreasing
    assert call([0.0] + good[1:-1] + [np.pi]) == -1        # pole rings
    assert call(good[:4] + good[3:7]) == -1                # a repeated colatitude
    assert call(good[:-1] + [float("nan")]) == -1          # not finite
    assert call(good, kappa=(-1.0,)) == -1                 # kappa <= 0
    assert call(good, kappa=(3.0, 3.0000000001)) == -2     # near-equal kappa
    assert not out.value


def test_batch_output_checks_without_gpu():
    """The binding checks each batch output against its request before any call: count, tensor,
    pinned or device memory, dtype, contiguity, length."""
    import torch
    from paper_1709_10314_gb300.smerf import _check_batch_outs
    needs = [(torch.float32, 12), (torch.float64, 6)]
    ok = [torch.zeros(12), torch.zeros(6, dtype=torch.float64)]
    for outs in (ok[:1],                                            # one output short of the requests
                 [ok[0], np.zeros(6)],                              # not a tensor
                 ok,                                                # pageable host memory
                 ):
        with pytest.raises(ValueError):
            _check_batch_outs(needs, outs)
    # the remaining checks come after the memory check; on a host without a GPU no tensor is
    # pinned, so they are reached with the memory check's answer fixed by a stand-in
    class Pinned(torch.Tensor):
        def is_pinned(self, *a, **k):
            return True
    pin = [o.as_subclass(Pinned) for o in ok]
    _check_batch_outs(needs, pin)
    for bad in ([pin[0], pin[1].float().as_subclass(Pinned)],       # dtype
                [pin[0], torch.zeros(5, dtype=torch.float64).as_subclass(Pinned)],  # too short
                [torch.zeros(12, 2)[:, 0].as_subclass(Pinned), pin[1]]):           # not contiguous
        with pytest.raises(ValueError):
            _check_batch_outs(needs, bad)


def test_khat_colatitude_validation_without_gpu(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.smerf_plan_create_khat_theta.restype = ctypes.c_int
    out = ctypes.c_void_p()
    good = [np.pi * (k + 0.5) / 8 for k in range(8)]

    def call(re, im, theta):
        r = np.ascontiguousarray(re, dtype=np.float64)
        i = np.ascontiguousarray(im, dtype=np.float64)
        t = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
        return lib.smerf_plan_create_khat_theta(r.ctypes.data_as(dp), i.ctypes.data_as(dp), len(re),
                                                ctypes.c_double(1.0), 8, None if t is None else t.ctypes.data_as(dp),
                                                32, ctypes.c_uint(0), 0, ctypes.byref(out))
    assert call([0.0, 0.0], [3.0, -3.0], None) == -1               # no colatitudes
    assert call([0.0, 0.0], [3.0, -3.0], good[::-1]) == -1         # decreasing
    assert call([0.0, 0.0], [3.0, -3.0], good[:-1] + [np.pi]) == -1  # a pole ring
    assert call([4.0], [0.0], good[:-1] + [np.pi]) == -1           # real kappa-hat: the same rules
    assert call([0.0, 0.0], [3.0, 2.0], good) == -1                # not a conjugate pair
    assert not out.value


def test_plan_spectrum_arguments_without_gpu(lib):
    from paper_1709_10314_gb300 import Plan
    with pytest.raises(ValueError):
        Plan(A=1.0, n_theta=8, n_phi=32)                             # no spectrum
    with pytest.raises(ValueError):
        Plan([3.0], 1.0, 8, 32, khat=[9.0])                          # two spectra
    with pytest.raises(ValueError):
        Plan([3.0], 1.0, 8, 32, theta=[0.5, 1.0, 1.5])               # not n_theta colatitudes


def test_plan_colatitudes_through_the_binding_without_gpu(lib):
    """The binding's calls of the two colatitude entry points marshal their arguments; the
    library rejects the colatitudes before it touches a GPU."""
    from paper_1709_10314_gb300 import Plan, SmerfError
    bad = [0.5, 0.4, 1.0, 1.5]                                        # not increasing
    for kw in (dict(kappa=[3.0]), dict(khat=[complex(0, 3), complex(0, -3)]), dict(khat=[9.0])):
        with pytest.raises(SmerfError) as e:
            Plan(A=1.0, n_theta=4, n_phi=32, theta=bad, **kw)
        assert e.value.status == -1


def test_null_handles_and_empty_calls_without_gpu(lib):
    """Every entry point that takes a plan or a batch answers SMERF_EINVAL for a NULL handle, and
    the empty calls are no-ops, before any CUDA call."""
    V = ctypes.c_void_p
    null = V()
    for fn, args in [
        ("smerf_sample", (null, ctypes.c_uint64(0), 1, null, null)),
        ("smerf_sample_timed", (null, ctypes.c_uint64(0), 1, null, null, null, null)),
        ("smerf_sample_host", (null, ctypes.c_uint64(0), 1, null, null)),
        ("smerf_sample_noalloc", (null, ctypes.c_uint64(0), 1, null, null)),
        ("smerf_sample_batched", (null, null, null, null, 1, null)),
        ("smerf_plan_info", (null, null)),
        ("smerf_plan_set_rings", (null, null, null)),
        ("smerf_plan_autotune", (null, 1, null, null)),
        ("smerf_plan_set_launch", (null, null)),
        ("smerf_plan_launch_candidates", (null, null, 0)),
        ("smerf_plan_copy_tables", (null, 0, 0, 0, null)),
        ("smerf_plan_create_many", (null, 1, null)),
        ("smerf_batch_create", (null, null, 1, ctypes.byref(V()))),
        ("smerf_batch_create", (null, null, 0, null)),
        ("smerf_batch_set", (null, null, null)),
        ("smerf_batch_launch", (null, null)),
        ("smerf_batch_sample", (null, null, null, null)),
        ("smerf_batch_info", (null, null, null)),
        ("smerf_batch_launch_count", (null,)),
        ("smerf_batch_status", (null, null)),
        ("smerf_batch_set_single_launch", (null, 0)),
        ("smerf_debug_batch_fail_waits", (null,)),
        ("smerf_philox_uint32", (ctypes.c_uint64(0), 0, ctypes.c_int64(-1), null, null)),
        ("smerf_ring_normals", (ctypes.c_uint64(0), 0, ctypes.c_int64(-1), 0, null, null)),
    ]:
        f = getattr(lib, fn)
        f.restype = ctypes.c_int
        assert f(*args) == -1, fn
    chosen = ctypes.c_int(7)
    cand = (ctypes.c_int * 1)(8)
    lib.smerf_plan_autotune_anchor.restype = ctypes.c_int
    assert lib.smerf_plan_autotune_anchor(null, 1, cand, 1, null, ctypes.byref(chosen)) == -1 and chosen.value == 0
    for fn, args in [
        ("smerf_sample_batched", (null, null, null, null, 0, null)),   # no requests
        ("smerf_plan_create_many", (null, 0, null)),                   # no plans
        ("smerf_batch_destroy", (null,)),
        ("smerf_philox_uint32", (ctypes.c_uint64(0), 0, ctypes.c_int64(0), null, null)),
        ("smerf_ring_normals", (ctypes.c_uint64(0), 0, ctypes.c_int64(0), 0, null, null)),
    ]:
        f = getattr(lib, fn)
        f.restype = ctypes.c_int
        assert f(*args) == 0, fn


def test_host_output_checks_without_gpu():
    """sample_host's buffer check: dtype, layout, writeability, memory kind and length."""
    import torch
    from paper_1709_10314_gb300.smerf import _check_host_out
    f32 = (np.float32, torch.float32, 12)
    _check_host_out(np.zeros(12, dtype=np.float32), *f32)
    _check_host_out(torch.zeros(3, 4), *f32)
    ro = np.zeros(12, dtype=np.float32)
    ro.flags.writeable = False
    for bad in (np.zeros(12), np.zeros(11, dtype=np.float32), np.zeros((12, 2), dtype=np.float32)[:, 0], ro,
                torch.zeros(12, dtype=torch.float64), torch.zeros(11), torch.zeros(12, 2)[:, 0], [0.0] * 12):
        with pytest.raises(ValueError):
            _check_host_out(bad, *f32)


def test_ring_layout_lengths_without_gpu():
    """set_rings takes one point count (and one offset) per ring; other lengths are refused before
    the library is called."""
    from paper_1709_10314_gb300 import Plan
    pl = Plan.__new__(Plan)  # no device tables: the check comes first
    pl.n_theta = 4
    pl.ring_points = None
    for args in (([8, 8, 8],), ([8] * 5,), ([8] * 4, [0.0] * 3)):
        with pytest.raises(ValueError):
            pl.set_rings(*args)
    assert pl.ring_points is None
