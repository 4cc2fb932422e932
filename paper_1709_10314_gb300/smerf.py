"""ctypes binding of the C ABI declared in include/smerf.h (argument marshalling only).

Names follow the C entry points: ``Plan`` wraps smerf_plan_create_ex / smerf_plan_info /
smerf_plan_copy_tables / smerf_sample / smerf_sample_host / smerf_plan_destroy.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libsmerf.so")

SMERF_RECUR_FP64 = 0x1
SMERF_TABLES_FP64 = 0x2
SMERF_TABLES_FP32 = 0x4
SMERF_ORDER_PAPER = 0x8


class SmerfError(RuntimeError):
    def __init__(self, call, status):
        self.status = status
        msg = _lib().smerf_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__("%s failed: %s (%d)" % (call, msg, status))


class _Info(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("n_modes", ctypes.c_int), ("start_ring", ctypes.c_int),
                ("chain_len", ctypes.c_int * 2), ("anchor_spacing", ctypes.c_int),
                ("n_anchors", ctypes.c_int * 2), ("n_segments", ctypes.c_int),
                ("flags", ctypes.c_uint), ("table_bytes", ctypes.c_size_t),
                ("scratch_bytes_per_sample", ctypes.c_size_t), ("setup_ms", ctypes.c_double),
                ("step_table_bytes", ctypes.c_size_t), ("points_per_sample", ctypes.c_size_t)]


_LIB = None
LAUNCH_INTS = 6  # SMERF_LAUNCH_INTS


def library_path():
    return _LIBPATH


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(_LIBPATH):
            raise ImportError("libsmerf.so is not built: run `python -m paper_1709_10314_gb300.build` "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(_LIBPATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        L.smerf_plan_create_ex.argtypes = [dp, ip, ctypes.c_double, ip, ip, ctypes.c_uint, ip,
                                           ctypes.POINTER(vp)]
        L.smerf_plan_create_ex.restype = ip
        L.smerf_plan_create_khat.argtypes = [dp, dp, ip, ctypes.c_double, ip, ip, ctypes.c_uint, ip, ctypes.POINTER(vp)]
        L.smerf_plan_create_theta.argtypes = [dp, ip, ctypes.c_double, ip, dp, ip, ctypes.c_uint, ip, ctypes.POINTER(vp)]
        L.smerf_plan_create_theta.restype = ip
        L.smerf_plan_create_khat.restype = ip
        L.smerf_plan_create_khat_theta.argtypes = [dp, dp, ip, ctypes.c_double, ip, dp, ip, ctypes.c_uint, ip,
                                                   ctypes.POINTER(vp)]
        L.smerf_plan_create_khat_theta.restype = ip
        L.smerf_plan_destroy.argtypes = [vp]
        L.smerf_plan_destroy.restype = ip
        L.smerf_sample.argtypes = [vp, ctypes.c_uint64, ip, vp, vp]
        L.smerf_sample.restype = ip
        L.smerf_sample_timed.argtypes = [vp, ctypes.c_uint64, ip, vp, vp, vp, vp]
        L.smerf_sample_timed.restype = ip
        L.smerf_sample_noalloc.argtypes = [vp, ctypes.c_uint64, ip, vp, vp]
        L.smerf_sample_noalloc.restype = ip
        L.smerf_plan_create_many.argtypes = [ctypes.POINTER(_PlanSpec), ip, ctypes.POINTER(vp)]
        L.smerf_plan_create_many.restype = ip
        L.smerf_last_device_status.argtypes = [vp]
        L.smerf_last_device_status.restype = ip
        L.smerf_scratch_trim.argtypes = []
        L.smerf_scratch_trim.restype = ip
        L.smerf_sample_launches.argtypes = [vp, ip]
        L.smerf_sample_launches.restype = ip
        L.smerf_sample_host.argtypes = [vp, ctypes.c_uint64, ip, vp, vp]
        L.smerf_sample_host.restype = ip
        L.smerf_sample_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ip), ctypes.POINTER(vp), ip, vp]
        L.smerf_sample_batched.restype = ip
        L.smerf_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ip), ip, ctypes.POINTER(vp)]
        L.smerf_batch_create.restype = ip
        L.smerf_batch_set.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(vp)]
        L.smerf_batch_set.restype = ip
        L.smerf_batch_launch.argtypes = [vp, vp]
        L.smerf_batch_launch.restype = ip
        L.smerf_batch_sample.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(vp), vp]
        L.smerf_batch_sample.restype = ip
        L.smerf_batch_info.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
        L.smerf_batch_info.restype = ip
        L.smerf_batch_launch_count.argtypes = [vp]
        L.smerf_batch_launch_count.restype = ip
        L.smerf_batch_status.argtypes = [vp, vp]
        L.smerf_batch_status.restype = ip
        L.smerf_batch_set_single_launch.argtypes = [vp, ip]
        L.smerf_batch_set_single_launch.restype = ip
        L.smerf_debug_batch_fail_waits.argtypes = [vp]
        L.smerf_debug_batch_fail_waits.restype = ip
        L.smerf_batch_destroy.argtypes = [vp]
        L.smerf_batch_destroy.restype = ip
        L.smerf_plan_info.argtypes = [vp, ctypes.POINTER(_Info)]
        L.smerf_plan_info.restype = ip
        L.smerf_plan_set_rings.argtypes = [vp, ctypes.POINTER(ip), dp]
        L.smerf_plan_set_rings.restype = ip
        L.smerf_plan_copy_tables.argtypes = [vp, ip, ip, ip, dp]
        L.smerf_plan_copy_tables.restype = ip
        L.smerf_plan_autotune.argtypes = [vp, ip, vp, ctypes.POINTER(ip)]
        L.smerf_plan_autotune.restype = ip
        L.smerf_plan_autotune_anchor.argtypes = [vp, ip, ctypes.POINTER(ip), ip, vp, ctypes.POINTER(ip)]
        L.smerf_plan_autotune_anchor.restype = ip
        L.smerf_plan_launch_candidates.argtypes = [vp, ctypes.POINTER(ip), ip]
        L.smerf_plan_launch_candidates.restype = ip
        L.smerf_plan_set_launch.argtypes = [vp, ctypes.POINTER(ip)]
        L.smerf_plan_set_launch.restype = ip
        L.smerf_philox_uint32.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, vp, vp]
        L.smerf_philox_uint32.restype = ip
        L.smerf_ring_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ip, vp, vp]
        L.smerf_ring_normals.restype = ip
        L.smerf_debug_fail_alloc.argtypes = [ip]
        L.smerf_debug_fail_alloc.restype = ip
        L.smerf_status_string.argtypes = [ip]
        L.smerf_status_string.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def _check(call, status):
    if status != 0:
        raise SmerfError(call, status)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class _PlanSpec(ctypes.Structure):
    _fields_ = [("kappa", ctypes.POINTER(ctypes.c_double)), ("p", ctypes.c_int), ("A", ctypes.c_double),
                ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int), ("flags", ctypes.c_uint),
                ("anchor_spacing", ctypes.c_int)]


class Plan:
    """A sampling plan (device-resident conditional-covariance tables)."""

    def __init__(self, kappa=None, A=1.0, n_theta=64, n_phi=128, flags=0, anchor_spacing=0, khat=None, theta=None):
        """Spectrum C_l = A / prod_i (l(l+1) + kappa-hat_i): real `kappa` (kappa-hat_i =
        kappa_i^2), or `khat` given directly (positive real values and adjacent complex-conjugate
        pairs, e.g. [a + ib, a - ib] or [a + ib, a - ib, c]).  `theta`: the ring colatitudes of
        another iso-latitude grid (smerf_plan_create_theta, smerf_plan_create_khat_theta), e.g.
        HEALPix or a band of latitudes."""
        L = _lib()
        h = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        if (kappa is None) == (khat is None):
            raise ValueError("give the spectrum as kappa or as khat")
        th = None
        if theta is not None:
            th = np.ascontiguousarray(theta, dtype=np.float64)
            if th.shape != (int(n_theta),):
                raise ValueError("theta must hold n_theta colatitudes")
        if khat is not None:
            kh = [complex(v) for v in np.atleast_1d(khat)]
            re = np.ascontiguousarray([v.real for v in kh], dtype=np.float64)
            im = np.ascontiguousarray([v.imag for v in kh], dtype=np.float64)
            if th is None:
                _check("smerf_plan_create_khat",
                       L.smerf_plan_create_khat(re.ctypes.data_as(dp), im.ctypes.data_as(dp), len(kh), float(A),
                                                int(n_theta), int(n_phi), int(flags), int(anchor_spacing),
                                                ctypes.byref(h)))
            else:
                _check("smerf_plan_create_khat_theta",
                       L.smerf_plan_create_khat_theta(re.ctypes.data_as(dp), im.ctypes.data_as(dp), len(kh),
                                                      float(A), int(n_theta), th.ctypes.data_as(dp), int(n_phi),
                                                      int(flags), int(anchor_spacing), ctypes.byref(h)))
            k = np.asarray(kh)
        elif th is not None:
            k = np.ascontiguousarray(np.atleast_1d(kappa), dtype=np.float64)
            _check("smerf_plan_create_theta",
                   L.smerf_plan_create_theta(k.ctypes.data_as(dp), len(k), float(A), int(n_theta),
                                             th.ctypes.data_as(dp), int(n_phi), int(flags), int(anchor_spacing),
                                             ctypes.byref(h)))
        else:
            k = np.ascontiguousarray(np.atleast_1d(kappa), dtype=np.float64)
            _check("smerf_plan_create_ex",
                   L.smerf_plan_create_ex(k.ctypes.data_as(dp), len(k),
                                          float(A), int(n_theta), int(n_phi), int(flags),
                                          int(anchor_spacing), ctypes.byref(h)))
        self._h = h
        self.kappa = k
        self.A = float(A)
        self.n_theta = int(n_theta)
        self.n_phi = int(n_phi)
        self.flags = int(flags)
        self.fp64 = bool(flags & SMERF_RECUR_FP64)
        self.ring_points = None

    def set_rings(self, n_phi_ring=None, phi0_ring=None):
        """smerf_plan_set_rings: ring k holds n_phi_ring[k] points from phi0_ring[k] (None: the
        full grid again).  sample() then returns [n_samples][sum(n_phi_ring)], rings back to back."""
        if n_phi_ring is None:
            _check("smerf_plan_set_rings", _lib().smerf_plan_set_rings(self._h, None, None))
            self.ring_points = None
            return
        if len(n_phi_ring) != self.n_theta or (phi0_ring is not None and len(phi0_ring) != self.n_theta):
            raise ValueError("one point count (and one offset) per ring: %d rings" % self.n_theta)
        n = (ctypes.c_int * self.n_theta)(*[int(v) for v in n_phi_ring])
        p0 = None if phi0_ring is None else (ctypes.c_double * self.n_theta)(*[float(v) for v in phi0_ring])
        _check("smerf_plan_set_rings", _lib().smerf_plan_set_rings(self._h, n, p0))
        self.ring_points = [int(v) for v in n_phi_ring]

    @property
    def points(self):
        """Output values of one realisation."""
        return sum(self.ring_points) if self.ring_points else self.n_theta * self.n_phi

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().smerf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self):
        inf = _Info()
        _check("smerf_plan_info", _lib().smerf_plan_info(self._h, ctypes.byref(inf)))
        return {"p": inf.p, "n_theta": inf.n_theta, "n_phi": inf.n_phi, "n_modes": inf.n_modes,
                "start_ring": inf.start_ring, "chain_len": list(inf.chain_len),
                "anchor_spacing": inf.anchor_spacing, "n_anchors": list(inf.n_anchors),
                "n_segments": inf.n_segments, "flags": inf.flags, "table_bytes": inf.table_bytes,
                "scratch_bytes_per_sample": inf.scratch_bytes_per_sample, "setup_ms": inf.setup_ms,
                "step_table_bytes": inf.step_table_bytes, "points_per_sample": inf.points_per_sample}

    def launches(self, n_samples):
        """smerf_sample_launches: kernels one sample() call of n_samples launches."""
        v = _lib().smerf_sample_launches(self._h, int(n_samples))
        if v < 0:
            _check("smerf_sample_launches", v)
        return v

    def autotune(self, n_samples, stream=None):
        """smerf_plan_autotune: returns (units/thread, realisations/CTA, producer threads, FFT
        threads, CTAs per SM)."""
        ch = (ctypes.c_int * LAUNCH_INTS)()
        _check("smerf_plan_autotune", _lib().smerf_plan_autotune(self._h, int(n_samples), _stream_ptr(stream), ch))
        return tuple(ch)

    def autotune_anchor(self, n_samples, candidates=(8, 12, 16, 24, 32), stream=None):
        """smerf_plan_autotune_anchor: rebuild the tables for each anchor spacing, keep the fastest;
        returns the chosen spacing (0 for a plan in Alg. 2's order)."""
        cand = (ctypes.c_int * len(candidates))(*[int(v) for v in candidates])
        ch = ctypes.c_int()
        _check("smerf_plan_autotune_anchor", _lib().smerf_plan_autotune_anchor(
            self._h, int(n_samples), cand, len(candidates), _stream_ptr(stream), ctypes.byref(ch)))
        return ch.value

    def launch_candidates(self):
        """smerf_plan_launch_candidates: list of (units/thread, realisations/CTA, producer
        threads, FFT threads, CTAs per SM, FFT radix plan 16 or 4)."""
        cap = 128
        buf = (ctypes.c_int * (LAUNCH_INTS * cap))()
        n = _lib().smerf_plan_launch_candidates(self._h, buf, cap)
        if n < 0:
            _check("smerf_plan_launch_candidates", n)
        return [tuple(buf[LAUNCH_INTS * i:LAUNCH_INTS * i + LAUNCH_INTS]) for i in range(min(n, cap))]

    def set_launch(self, config):
        """smerf_plan_set_launch: fix a launch configuration (None: built-in choice)."""
        if config is None:
            ptr = None
        else:
            if len(config) != LAUNCH_INTS:
                raise ValueError("a launch configuration has %d integers" % LAUNCH_INTS)
            ptr = (ctypes.c_int * LAUNCH_INTS)(*[int(v) for v in config])
        _check("smerf_plan_set_launch", _lib().smerf_plan_set_launch(self._h, ptr))

    def tables(self, which, chain=0, pos=0):
        """Copy a table block to host as float64 [rows][n_modes] (see smerf_plan_copy_tables)."""
        p = len(self.kappa)
        rows = {0: p * (p + 1) // 2, 1: 2 * p * p + p * (p + 1) // 2, 2: p * p + p * (p + 1) // 2}[which]
        out = np.zeros((rows, self.n_phi // 2 + 1))
        _check("smerf_plan_copy_tables",
               _lib().smerf_plan_copy_tables(self._h, which, chain, pos,
                                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.fp64 else torch.float32

    def _check_out(self, out, n_samples):
        """The C ABI cannot see a buffer's length: a device tensor of this plan's dtype, dense,
        on the current device, with room for n_samples realisations, or ValueError."""
        import torch
        if not isinstance(out, torch.Tensor) or not out.is_cuda:
            raise ValueError("out must be a CUDA tensor")
        if out.dtype != self.dtype:
            raise ValueError("out has dtype %s; this plan writes %s" % (out.dtype, self.dtype))
        if not out.is_contiguous():
            raise ValueError("out must be contiguous")
        if out.device.index != torch.cuda.current_device():
            raise ValueError("out is on %s, the current device is cuda:%d" % (out.device, torch.cuda.current_device()))
        if int(n_samples) < 0 or out.numel() < int(n_samples) * self.points:
            raise ValueError("out holds %d elements; %d realisations need %d" % (
                out.numel(), int(n_samples), int(n_samples) * self.points))

    def sample(self, seed, n_samples, out=None, stream=None):
        """Device realisations [n_samples][n_theta][n_phi] (torch tensor on the current device)."""
        import torch
        if out is None:
            shape = (n_samples, self.points) if self.ring_points else (n_samples, self.n_theta, self.n_phi)
            out = torch.empty(shape, dtype=self.dtype, device="cuda")
        self._check_out(out, n_samples)
        _check("smerf_sample", _lib().smerf_sample(self._h, ctypes.c_uint64(seed & (2**64 - 1)), int(n_samples),
                                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def sample_noalloc(self, seed, n_samples, out, stream=None):
        """smerf_sample_noalloc: like sample() but the library allocates nothing (its scratch
        is a fixed 16 MiB device array; larger requests raise SmerfError SMERF_ESCRATCH)."""
        self._check_out(out, n_samples)
        _check("smerf_sample_noalloc",
               _lib().smerf_sample_noalloc(self._h, ctypes.c_uint64(seed & (2**64 - 1)), int(n_samples),
                                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def sample_timed(self, seed, n_samples, out, ev_before, ev_after, stream=None):
        """smerf_sample_timed: records the two torch.cuda.Event objects around the segment kernel."""
        self._check_out(out, n_samples)
        for ev in (ev_before, ev_after):
            if not ev.cuda_event:
                ev.record()  # torch creates the event handle lazily
        _check("smerf_sample_timed",
               _lib().smerf_sample_timed(self._h, ctypes.c_uint64(seed & (2**64 - 1)), int(n_samples),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream),
                                         ctypes.c_void_p(ev_before.cuda_event), ctypes.c_void_p(ev_after.cuda_event)))
        return out

    def sample_host(self, seed, n_samples, out=None, stream=None):
        """Realisations into host memory (numpy array or pinned torch CPU tensor)."""
        dt = np.float64 if self.fp64 else np.float32
        if out is None:
            shape = (n_samples, self.points) if self.ring_points else (n_samples, self.n_theta, self.n_phi)
            out = np.empty(shape, dtype=dt)
        if int(n_samples) < 0:
            raise ValueError("n_samples must be >= 0")
        _check_host_out(out, dt, self.dtype, int(n_samples) * self.points)
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        _check("smerf_sample_host", _lib().smerf_sample_host(self._h, ctypes.c_uint64(seed & (2**64 - 1)),
                                                              int(n_samples), ctypes.c_void_p(ptr),
                                                              _stream_ptr(stream)))
        return out


def create_plans(specs):
    """smerf_plan_create_many: Plans for a list of dicts with the keys of Plan(kappa, A, n_theta,
    n_phi, flags, anchor_spacing), their set-ups overlapping on the GPU."""
    n = len(specs)
    ks = [np.ascontiguousarray(np.atleast_1d(d["kappa"]), dtype=np.float64) for d in specs]
    arr = (_PlanSpec * max(n, 1))()
    dp = ctypes.POINTER(ctypes.c_double)
    for i, (d, k) in enumerate(zip(specs, ks)):
        arr[i] = _PlanSpec(k.ctypes.data_as(dp), len(k), float(d.get("A", 1.0)), int(d["n_theta"]),
                           int(d["n_phi"]), int(d.get("flags", 0)), int(d.get("anchor_spacing", 0)))
    hs = (ctypes.c_void_p * max(n, 1))()
    _check("smerf_plan_create_many", _lib().smerf_plan_create_many(arr, n, hs))
    plans = []
    for i, (d, k) in enumerate(zip(specs, ks)):
        pl = Plan.__new__(Plan)
        pl._h = ctypes.c_void_p(hs[i])
        pl.kappa = k
        pl.A = float(d.get("A", 1.0))
        pl.n_theta = int(d["n_theta"])
        pl.n_phi = int(d["n_phi"])
        pl.flags = int(d.get("flags", 0))
        pl.fp64 = bool(pl.flags & SMERF_RECUR_FP64)
        pl.ring_points = None
        plans.append(pl)
    return plans


def last_device_status(stream=None):
    """smerf_last_device_status: synchronise the stream and return 0 or SMERF_ECUDA."""
    return _lib().smerf_last_device_status(_stream_ptr(stream))


def debug_fail_alloc(k):
    """smerf_debug_fail_alloc: make the allocation after k more fail (k < 0: off)."""
    _check("smerf_debug_fail_alloc", _lib().smerf_debug_fail_alloc(int(k)))


def scratch_trim():
    """smerf_scratch_trim: release the idle memory of the per-call scratch pool (current device)."""
    _check("smerf_scratch_trim", _lib().smerf_scratch_trim())


def _check_host_out(out, np_dtype, torch_dtype, need):
    """The C ABI cannot see a buffer's length: a host output is a writeable C-contiguous numpy
    array of np_dtype, or a contiguous CPU torch tensor of torch_dtype, holding at least `need`
    elements; else ValueError."""
    import torch
    if isinstance(out, np.ndarray):
        if out.dtype != np_dtype:
            raise ValueError("out has dtype %s; this plan writes %s" % (out.dtype, np.dtype(np_dtype)))
        if not out.flags["C_CONTIGUOUS"] or not out.flags["WRITEABLE"]:
            raise ValueError("out must be a writeable C-contiguous array")
        n = out.size
    elif isinstance(out, torch.Tensor):
        if out.is_cuda:
            raise ValueError("out is a CUDA tensor; sample() writes device memory")
        if out.dtype != torch_dtype:
            raise ValueError("out has dtype %s; this plan writes %s" % (out.dtype, torch_dtype))
        if not out.is_contiguous():
            raise ValueError("out must be contiguous")
        n = out.numel()
    else:
        raise ValueError("out must be a numpy array or a CPU torch tensor")
    if n < need:
        raise ValueError("out holds %d elements; the realisations need %d" % (n, need))


def _batch_needs(plans, n_samples):
    """(dtype, elements) that each request's output must hold."""
    return [(p.dtype, int(n) * p.points) for p, n in zip(plans, n_samples)]


def _check_batch_outs(needs, outs):
    """The C ABI cannot see a buffer's length.  Request i's output: a tensor of its plan's dtype,
    dense, with room for its realisations (needs[i] = (dtype, elements)), on the current CUDA
    device or in page-locked host memory (which the kernels write over the CPU-GPU link); else
    ValueError."""
    import torch
    if len(outs) != len(needs):
        raise ValueError("%d outputs for %d requests" % (len(outs), len(needs)))
    cur = None
    for i, ((dt, need), o) in enumerate(zip(needs, outs)):
        if not isinstance(o, torch.Tensor):
            raise ValueError("output %d is not a tensor" % i)
        if o.is_cuda:
            cur = torch.cuda.current_device() if cur is None else cur
            if o.device.index != cur:
                raise ValueError("output %d is on %s, the current device is cuda:%d" % (i, o.device, cur))
        elif not o.is_pinned():
            raise ValueError("output %d is in pageable host memory; use a CUDA or pinned tensor" % i)
        if o.dtype != dt:
            raise ValueError("output %d has dtype %s; its plan writes %s" % (i, o.dtype, dt))
        if not o.is_contiguous():
            raise ValueError("output %d must be contiguous" % i)
        if o.numel() < need:
            raise ValueError("output %d holds %d elements; its realisations need %d" % (i, o.numel(), need))


def sample_batched(plans, seeds, n_samples, outs, stream=None):
    if len(n_samples) != len(plans) or len(seeds) != len(plans) or min([int(v) for v in n_samples] + [0]) < 0:
        raise ValueError("one seed and one count >= 0 per plan")
    _check_batch_outs(_batch_needs(plans, n_samples), outs)
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    S = (ctypes.c_uint64 * n)(*[s & (2**64 - 1) for s in seeds])
    N = (ctypes.c_int * n)(*[int(v) for v in n_samples])
    O = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check("smerf_sample_batched", _lib().smerf_sample_batched(P, S, N, O, n, _stream_ptr(stream)))
    return outs


class Batch:
    """A reusable batch (smerf_batch_create / _set / _launch / _sample / _info / _destroy)."""

    def __init__(self, plans, n_samples):
        L = _lib()
        n = len(plans)
        self._plans = list(plans)  # keep the plans alive
        self.n_samples = [int(v) for v in n_samples]
        if len(self.n_samples) != n:
            raise ValueError("%d counts for %d plans" % (len(self.n_samples), n))
        P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
        N = (ctypes.c_int * n)(*self.n_samples)
        h = ctypes.c_void_p()
        _check("smerf_batch_create", L.smerf_batch_create(P, N, n, ctypes.byref(h)))
        self._h = h
        self._needs = _batch_needs(plans, self.n_samples)  # the ring layouts the batch was made with

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().smerf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, seeds, outs):
        if len(seeds) != len(self._plans):
            raise ValueError("%d seeds for %d requests" % (len(seeds), len(self._plans)))
        _check_batch_outs(self._needs, outs)
        n = len(self._plans)
        S = (ctypes.c_uint64 * n)(*[s & (2**64 - 1) for s in seeds])
        O = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        return S, O

    def set(self, seeds, outs):
        S, O = self._arrays(seeds, outs)
        _check("smerf_batch_set", _lib().smerf_batch_set(self._h, S, O))

    def launch(self, stream=None):
        _check("smerf_batch_launch", _lib().smerf_batch_launch(self._h, _stream_ptr(stream)))

    def sample(self, seeds, outs, stream=None):
        S, O = self._arrays(seeds, outs)
        _check("smerf_batch_sample", _lib().smerf_batch_sample(self._h, S, O, _stream_ptr(stream)))
        return outs

    def set_single_launch(self, single):
        """smerf_batch_set_single_launch: True runs the FP32-recursion work of the following launches
        as one persistent launch (anchor items, then segment items), False (the default) as an
        anchor launch and a persistent launch."""
        _check("smerf_batch_set_single_launch", _lib().smerf_batch_set_single_launch(self._h, 1 if single else 0))

    def status(self, stream=None):
        """smerf_batch_status: synchronises the stream; SMERF_OK (0), or SMERF_ETIMEOUT (-7) when a
        segment item's wait for its request's anchors ran out in the last launch."""
        return _lib().smerf_batch_status(self._h, _stream_ptr(stream))

    def debug_fail_waits(self):
        """smerf_debug_batch_fail_waits: the next launch's anchor waits cannot be met (test hook)."""
        _check("smerf_debug_batch_fail_waits", _lib().smerf_debug_batch_fail_waits(self._h))

    def info(self):
        g, s1 = ctypes.c_int(), ctypes.c_int()
        _check("smerf_batch_info", _lib().smerf_batch_info(self._h, ctypes.byref(g), ctypes.byref(s1)))
        return {"groups": g.value, "singles": s1.value, "launches": _lib().smerf_batch_launch_count(self._h)}


def philox_uint32(key64, ring, ncalls, stream=None):
    import torch
    out = torch.empty(4 * ncalls, dtype=torch.int32, device="cuda")
    _check("smerf_philox_uint32", _lib().smerf_philox_uint32(ctypes.c_uint64(key64 & (2**64 - 1)), ring,
                                                              ncalls, ctypes.c_void_p(out.data_ptr()),
                                                              _stream_ptr(stream)))
    return out


def ring_normals(key64, ring, n, fp64=False, stream=None):
    import torch
    out = torch.empty(n, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    _check("smerf_ring_normals", _lib().smerf_ring_normals(ctypes.c_uint64(key64 & (2**64 - 1)), ring, n,
                                                            int(bool(fp64)), ctypes.c_void_p(out.data_ptr()),
                                                            _stream_ptr(stream)))
    return out
