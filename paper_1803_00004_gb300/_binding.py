"""ctypes binding of include/bf.h (argument marshalling only).

Every computation happens in libbf.so; this module converts Python values and
PyTorch CUDA tensors (data pointer, row pitch, current stream) into the C ABI's
plain pointers and sizes.  If the library has not been built, every entry point
raises ``RuntimeError``: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libbf.so")

# ---- enums (mirrors include/bf.h)
OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_ADMISSION = 1, 2, 3, 4, 5
ERR_TIMEOUT, ERR_DEVICE_TIMEOUT, ERR_RANGE, ERR_NO_DEVICE, ERR_NOT_FOUND, ERR_CANCELLED = 6, 7, 8, 9, 10, 11
ERR_SCRATCH = 12
KERNEL_GAUSSIAN, KERNEL_EXPONENTIAL, KERNEL_BOX = 0, 1, 2
RANGE_TRUNCATED_MIN_PERIOD, RANGE_UNTRUNCATED_FULL, RANGE_PAPER_3D = 0, 1, 2
SERIES_COSINE, SERIES_HAAR = 0, 1
PREC_FP32, PREC_BF16, PREC_FP16 = 0, 1, 2


class bf_plan_desc(C.Structure):
    _fields_ = [("spatial", C.c_int), ("sigma_s", C.c_double), ("radius", C.c_int), ("ns_terms", C.c_int),
                ("range", C.c_int), ("sigma_r", C.c_double), ("t_r", C.c_double), ("nr_terms", C.c_int),
                ("policy", C.c_int), ("i_lo", C.c_float), ("i_hi", C.c_float), ("precision", C.c_int),
                ("kahan", C.c_int), ("device", C.c_int), ("z_bins", C.c_int), ("range_series", C.c_int)]


class bf_coeff_view(C.Structure):
    _fields_ = [("radius", C.c_int), ("t_s", C.c_double), ("haar_levels", C.c_int), ("t_r", C.c_double),
                ("period", C.c_double), ("nr", C.c_int), ("k", C.POINTER(C.c_int)), ("a", C.POINTER(C.c_double)),
                ("ns", C.c_int), ("haar_terms", C.POINTER(C.c_int)), ("haar_coef", C.POINTER(C.c_double)),
                ("tie_split", C.c_int), ("kernel", C.POINTER(C.c_double)), ("n_vwin", C.c_int),
                ("n_hwin", C.c_int), ("vwin", C.POINTER(C.c_int)), ("hwin", C.POINTER(C.c_int)),
                ("wcoef", C.POINTER(C.c_double)), ("range_max_err", C.c_double), ("spatial_max_err", C.c_double),
                ("den_eps", C.c_double), ("passes", C.c_int), ("z_bins", C.c_int), ("z_radius", C.c_int),
                ("range_series", C.c_int), ("n_range_haar", C.c_int), ("range_haar", C.POINTER(C.c_int)),
                ("range_haar_coef", C.POINTER(C.c_double)), ("z_weights", C.POINTER(C.c_double))]


class bf_image(C.Structure):
    _fields_ = [("d_in", C.c_void_p), ("in_pitch_bytes", C.c_size_t), ("d_out", C.c_void_p),
                ("out_pitch_bytes", C.c_size_t), ("height", C.c_int), ("width", C.c_int)]


class bf_serve_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int), ("n_streams", C.c_int),
                ("device", C.c_int), ("max_batch", C.c_int), ("plan_threads", C.c_int)]


MEM_DEVICE, MEM_HOST = 0, 1


class bf_request(C.Structure):
    _fields_ = [("desc", bf_plan_desc), ("in_", C.c_void_p), ("in_pitch_bytes", C.c_size_t), ("out", C.c_void_p),
                ("out_pitch_bytes", C.c_size_t), ("height", C.c_int), ("width", C.c_int), ("memory", C.c_int)]


class bf_result(C.Structure):
    _fields_ = [("status", C.c_int), ("latency_ns", C.c_uint64), ("queue_ns", C.c_uint64), ("plan_ns", C.c_uint64),
                ("device_ns", C.c_uint64)]

    # milliseconds, for convenience
    latency_ms = property(lambda self: self.latency_ns * 1e-6)
    queue_ms = property(lambda self: self.queue_ns * 1e-6)
    plan_ms = property(lambda self: self.plan_ns * 1e-6)
    device_ms = property(lambda self: self.device_ns * 1e-6)


EXPORTS = ["bf_plan_desc_default", "bf_plan_create", "bf_plan_destroy", "bf_coeffs", "bf_launch_info", "bf_autotune",
           "bf_autotune_group", "bf_autotune_image",
           "bf_launch_candidates", "bf_set_launch",
           "bf_filter", "bf_filter_noalloc",
           "bf_filter_batch", "bf_autotune_batch",
           "bf_exact", "bf_exact_lut", "bf_precompute", "bf_filter_cached", "bf_cache_bytes", "bf_cache_destroy",
           "bf_serve_create", "bf_serve_submit", "bf_serve_poll", "bf_serve_cancel", "bf_serve_destroy",
           "bf_status_string", "bf_last_error", "bf_version", "bf_debug_fail_launches", "bf_debug_range_checks",
           "bf_fp32_peak", "bf_filter_host"]

_lib = None
_lock = threading.Lock()


def lib():
    """Loads libbf.so (raises RuntimeError if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbf.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P, vp, sz, i, d = C.POINTER, C.c_void_p, C.c_size_t, C.c_int, C.c_double
        L.bf_plan_desc_default.argtypes = [P(bf_plan_desc)]
        L.bf_plan_desc_default.restype = None
        L.bf_plan_create.argtypes = [P(bf_plan_desc), P(vp)]
        L.bf_plan_destroy.argtypes = [vp]
        L.bf_plan_destroy.restype = None
        L.bf_coeffs.argtypes = [vp, P(bf_coeff_view)]
        L.bf_filter.argtypes = [vp, vp, sz, vp, sz, i, i, vp]
        L.bf_launch_info.argtypes = [vp, i, i, P(i)]
        L.bf_launch_candidates.argtypes = [vp, i, i, i, P(i), P(i)]
        L.bf_set_launch.argtypes = [vp, i, i, P(i)]
        L.bf_filter_noalloc.argtypes = [vp, vp, sz, vp, sz, i, i, vp]
        L.bf_autotune.argtypes = [vp, i, i, vp, P(i)]
        L.bf_autotune_group.argtypes = [P(vp), i, i, i, i, P(i)]
        L.bf_autotune_image.argtypes = [vp, vp, sz, i, i, vp, P(i)]
        L.bf_filter_batch.argtypes = [P(vp), P(bf_image), i, vp]
        L.bf_autotune_batch.argtypes = [P(vp), P(bf_image), i, vp]
        L.bf_exact.argtypes = [vp, sz, vp, sz, i, i, i, d, i, i, d, vp]
        L.bf_exact_lut.argtypes = [vp, sz, vp, sz, i, i, i, d, i, i, d, d, i, vp]
        L.bf_precompute.argtypes = [vp, vp, sz, i, i, i, i, vp, P(vp)]
        L.bf_filter_cached.argtypes = [vp, vp, vp, sz, vp, sz, vp]
        L.bf_cache_bytes.argtypes = [vp]
        L.bf_cache_bytes.restype = sz
        L.bf_cache_destroy.argtypes = [vp]
        L.bf_cache_destroy.restype = None
        L.bf_serve_create.argtypes = [P(bf_serve_config), P(vp)]
        L.bf_serve_submit.argtypes = [vp, P(bf_request), P(C.c_uint64)]
        L.bf_serve_poll.argtypes = [vp, C.c_uint64, i, P(bf_result)]
        L.bf_serve_cancel.argtypes = [vp, C.c_uint64]
        L.bf_serve_destroy.argtypes = [vp]
        L.bf_serve_destroy.restype = None
        L.bf_status_string.argtypes = [i]
        L.bf_status_string.restype = C.c_char_p
        L.bf_last_error.argtypes = []
        L.bf_last_error.restype = C.c_char_p
        L.bf_version.restype = i
        L.bf_debug_fail_launches.argtypes = [i]
        L.bf_debug_fail_launches.restype = None
        L.bf_debug_range_checks.argtypes = [i]
        L.bf_debug_range_checks.restype = None
        L.bf_fp32_peak.argtypes = [i, i, P(d), P(d)]
        L.bf_filter_host.argtypes = [P(vp), i, vp, sz, P(vp), sz, i, i, i, vp]
        _lib = L
    return _lib


class BFError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        self.status = status
        msg = L.bf_status_string(status).decode()
        detail = L.bf_last_error().decode()
        super().__init__("%s: %s%s" % (where, msg, (" (" + detail + ")") if detail else ""))


def _check(st: int, where: str) -> None:
    if st != OK:
        raise BFError(st, where)


def desc(**kw) -> bf_plan_desc:
    """A bf_plan_desc with the library defaults, overridden by keyword arguments."""
    d = bf_plan_desc()
    lib().bf_plan_desc_default(C.byref(d))
    for k, v in kw.items():
        if not hasattr(d, k):
            raise TypeError("unknown plan field %r" % k)
        setattr(d, k, v)
    return d


class Plan:
    """Owns a bf_plan*."""

    def __init__(self, d: bf_plan_desc | None = None, **kw):
        if d is None:
            d = desc(**kw)
        elif kw:
            raise TypeError("pass either a desc or keyword fields")
        self.desc = d
        h = C.c_void_p()
        _check(lib().bf_plan_create(C.byref(d), C.byref(h)), "bf_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().bf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coeffs(self) -> dict:
        return bf_coeffs(self)


def bf_coeffs(plan: Plan) -> dict:
    v = bf_coeff_view()
    _check(lib().bf_coeffs(plan.handle, C.byref(v)), "bf_coeffs")
    R = v.radius
    w = 2 * R + 1
    arr = lambda p, n: [p[j] for j in range(n)]
    return {
        "radius": R, "t_s": v.t_s, "haar_levels": v.haar_levels, "t_r": v.t_r, "period": v.period,
        "k": arr(v.k, v.nr), "a": arr(v.a, v.nr),
        "haar_terms": [tuple(v.haar_terms[4 * t + j] for j in range(4)) for t in range(v.ns)],
        "haar_coef": arr(v.haar_coef, v.ns), "tie_split": bool(v.tie_split),
        "kernel": [[v.kernel[r * w + c] for c in range(w)] for r in range(w)],
        "vwin": [(v.vwin[2 * j], v.vwin[2 * j + 1]) for j in range(v.n_vwin)],
        "hwin": [(v.hwin[2 * j], v.hwin[2 * j + 1]) for j in range(v.n_hwin)],
        "wcoef": [[v.wcoef[a * v.n_hwin + b] for b in range(v.n_hwin)] for a in range(v.n_vwin)],
        "range_max_err": v.range_max_err, "spatial_max_err": v.spatial_max_err, "den_eps": v.den_eps,
        "passes": v.passes, "z_bins": v.z_bins, "z_radius": v.z_radius, "range_series": v.range_series,
        "range_haar": [(v.range_haar[2 * t], v.range_haar[2 * t + 1]) for t in range(v.n_range_haar)],
        "range_haar_coef": arr(v.range_haar_coef, v.n_range_haar),
        "z_weights": arr(v.z_weights, 2 * v.z_radius + 1) if v.z_weights else [],
    }


INFO_KEYS = ("tw", "th", "threads", "nk", "groups", "launches", "smem", "scratch_kib", "ring", "depth", "ncols",
             "packed", "pre")


def bf_launch_info(plan: Plan, height: int, width: int) -> dict:
    info = (C.c_int * len(INFO_KEYS))()
    _check(lib().bf_launch_info(plan.handle, height, width, info), "bf_launch_info")
    keys = INFO_KEYS
    return dict(zip(keys, list(info)))


def bf_launch_candidates(plan: Plan, height: int, width: int, max_n: int = 4096) -> list:
    """Launch geometries for this plan and image size, best first by the cost model."""
    buf = (C.c_int * (len(INFO_KEYS) * max_n))()
    n = C.c_int(0)
    _check(lib().bf_launch_candidates(plan.handle, height, width, max_n, buf, C.byref(n)), "bf_launch_candidates")
    vals = list(buf)
    n_keys = len(INFO_KEYS)
    return [dict(zip(INFO_KEYS, vals[n_keys * k:n_keys * (k + 1)])) for k in range(n.value)]


def bf_set_launch(plan: Plan, height: int, width: int, info: dict) -> None:
    """Pins one geometry of bf_launch_candidates for later filter calls."""
    arr = (C.c_int * len(INFO_KEYS))(*[int(info[k]) for k in INFO_KEYS])
    _check(lib().bf_set_launch(plan.handle, height, width, arr), "bf_set_launch")


def bf_autotune(plan: Plan, height: int, width: int, stream=None) -> dict:
    info = (C.c_int * len(INFO_KEYS))()
    _check(lib().bf_autotune(plan.handle, height, width, _stream_handle(stream), info), "bf_autotune")
    keys = INFO_KEYS
    return dict(zip(keys, list(info)))


def bf_autotune_image(plan: Plan, src, stream=None) -> dict:
    """bf_autotune timed on the caller's image (a 2-D float32 device tensor)."""
    ip, ipitch, h, w = _ptr_pitch(src)
    info = (C.c_int * len(INFO_KEYS))()
    _check(lib().bf_autotune_image(plan.handle, ip, ipitch, h, w, _stream_handle(stream), info), "bf_autotune_image")
    return dict(zip(INFO_KEYS, list(info)))


def bf_autotune_group(plans, height: int, width: int, n_streams: int = 3) -> list:
    """Tunes the geometries of plans filtering concurrently (plan i on stream i mod n_streams) and pins
    them; returns each plan's geometry."""
    n = len(plans)
    hs = (C.c_void_p * max(n, 1))(*[p.handle for p in plans])
    infos = (C.c_int * (len(INFO_KEYS) * max(n, 1)))()
    _check(lib().bf_autotune_group(hs, n, height, width, n_streams, infos), "bf_autotune_group")
    k = len(INFO_KEYS)
    return [dict(zip(INFO_KEYS, list(infos[j * k:(j + 1) * k]))) for j in range(n)]


def _ptr_pitch(t):
    """(device pointer, row pitch in bytes, height, width) of a 2-D float32 tensor or a raw tuple."""
    if isinstance(t, tuple):
        return t
    if t.dim() != 2 or t.dtype.itemsize != 4 or t.stride(1) != 1:
        raise ValueError("expected a 2-D float32 tensor with unit column stride")
    return t.data_ptr(), t.stride(0) * 4, t.shape[0], t.shape[1]


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def bf_filter(plan: Plan, src, dst, stream=None) -> None:
    """Filters src into dst (CUDA float32 2-D tensors or (ptr, pitch, h, w) tuples)."""
    ip, ipitch, h, w = _ptr_pitch(src)
    op, opitch, h2, w2 = _ptr_pitch(dst)
    if (h, w) != (h2, w2):
        raise ValueError("input and output shapes differ")
    _check(lib().bf_filter(plan.handle, ip, ipitch, op, opitch, h, w, _stream_handle(stream)), "bf_filter")


def bf_filter_host(plans, src, dsts, n_streams: int = 3, stream=None) -> None:
    """Filters one host image (a 2-D float32 CPU tensor, pinned for asynchronous copies) with each plan into
    the host tensors dsts (same shape); asynchronous on `stream` (synchronize before reading dsts)."""
    n = len(plans)
    if len(dsts) != n:
        raise ValueError("one output per plan")
    for t in [src] + list(dsts):
        if t.dim() != 2 or t.dtype.itemsize != 4 or t.stride(1) != 1 or t.is_cuda:
            raise ValueError("expected 2-D float32 host tensors with unit column stride")
        if t.shape != src.shape or t.stride(0) != dsts[0].stride(0) and t is not src:
            raise ValueError("outputs must share the input's shape and one row pitch")
    hs = (C.c_void_p * n)(*[p.handle for p in plans])
    outs = (C.c_void_p * n)(*[t.data_ptr() for t in dsts])
    _check(lib().bf_filter_host(hs, n, src.data_ptr(), src.stride(0) * 4, outs, dsts[0].stride(0) * 4,
                                src.shape[0], src.shape[1], n_streams, _stream_handle(stream)), "bf_filter_host")


def _batch_args(plans, srcs, dsts):
    n = len(srcs)
    if len(plans) != n or len(dsts) != n:
        raise ValueError("plans, inputs and outputs must have the same length")
    imgs = (bf_image * max(n, 1))()
    hs = (C.c_void_p * max(n, 1))()
    for j in range(n):
        ip, ipitch, h, w = _ptr_pitch(srcs[j])
        op, opitch, h2, w2 = _ptr_pitch(dsts[j])
        if (h, w) != (h2, w2):
            raise ValueError("image %d: input and output shapes differ" % j)
        imgs[j] = bf_image(ip, ipitch, op, opitch, h, w)
        hs[j] = plans[j].handle
    return hs, imgs, n


def bf_filter_batch(plans, srcs, dsts, stream=None) -> None:
    hs, imgs, n = _batch_args(plans, srcs, dsts)
    _check(lib().bf_filter_batch(hs, imgs, n, _stream_handle(stream)), "bf_filter_batch")


def bf_autotune_batch(plans, srcs, dsts, stream=None) -> None:
    """Tunes the batched launch's geometry on this batch (bf_filter_batch's arguments); dsts receive results."""
    hs, imgs, n = _batch_args(plans, srcs, dsts)
    _check(lib().bf_autotune_batch(hs, imgs, n, _stream_handle(stream)), "bf_autotune_batch")


def bf_exact(src, dst, spatial=KERNEL_GAUSSIAN, sigma_s=4.0, radius=0, range=KERNEL_GAUSSIAN, sigma_r=0.1,
             stream=None) -> None:
    ip, ipitch, h, w = _ptr_pitch(src)
    op, opitch, _, _ = _ptr_pitch(dst)
    _check(lib().bf_exact(ip, ipitch, op, opitch, h, w, spatial, sigma_s, radius, range, sigma_r,
                          _stream_handle(stream)), "bf_exact")


def bf_exact_lut(src, dst, levels=256, data_range=1.0, spatial=KERNEL_GAUSSIAN, sigma_s=4.0, radius=0,
                 range=KERNEL_GAUSSIAN, sigma_r=0.1, stream=None) -> None:
    ip, ipitch, h, w = _ptr_pitch(src)
    op, opitch, _, _ = _ptr_pitch(dst)
    _check(lib().bf_exact_lut(ip, ipitch, op, opitch, h, w, spatial, sigma_s, radius, range, sigma_r, data_range,
                              levels, _stream_handle(stream)), "bf_exact_lut")


class Cache:
    """Owns a bf_cache* (the pre-computed window sums of one image, Sec. V-C, Case 1)."""

    def __init__(self, plan: "Plan", src, kmax: int, precision: int = 0, stream=None):
        ip, ipitch, h, w = _ptr_pitch(src)
        self.handle = C.c_void_p()
        _check(lib().bf_precompute(plan.handle, ip, ipitch, h, w, kmax, precision, _stream_handle(stream),
                                   C.byref(self.handle)), "bf_precompute")

    def filter(self, plan: "Plan", src, dst, stream=None) -> None:
        ip, ipitch, _, _ = _ptr_pitch(src)
        op, opitch, _, _ = _ptr_pitch(dst)
        _check(lib().bf_filter_cached(self.handle, plan.handle, ip, ipitch, op, opitch, _stream_handle(stream)),
               "bf_filter_cached")

    def nbytes(self) -> int:
        return int(lib().bf_cache_bytes(self.handle))

    def close(self) -> None:
        if self.handle:
            lib().bf_cache_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bf_version() -> int:
    return int(lib().bf_version())


def bf_fp32_peak(device: int = 0, iters: int = 20000) -> dict:
    """Measured fp32 lane operations per second of the scalar FFMA and the two-wide FFMA2."""
    a, b = C.c_double(), C.c_double()
    _check(lib().bf_fp32_peak(device, iters, C.byref(a), C.byref(b)), "bf_fp32_peak")
    return {"ffma_ops": a.value, "ffma2_ops": b.value}


def bf_debug_fail_launches(n: int) -> None:
    lib().bf_debug_fail_launches(int(n))


def bf_debug_range_checks(on: bool) -> None:
    lib().bf_debug_range_checks(1 if on else 0)


class Server:
    """Owns a bf_server* (continuous-batching request loop on one device)."""

    def __init__(self, hbm_budget_bytes=0, max_slots=0, n_streams=0, device=0, max_batch=0, plan_threads=0):
        cfg = bf_serve_config(hbm_budget_bytes, max_slots, n_streams, device, max_batch, plan_threads)
        h = C.c_void_p()
        _check(lib().bf_serve_create(C.byref(cfg), C.byref(h)), "bf_serve_create")
        self._h = h

    def submit(self, d: bf_plan_desc, in_ptr: int, out_ptr: int, height: int, width: int, in_pitch: int = 0,
               out_pitch: int = 0, memory: int = MEM_HOST) -> int:
        """Queues a request; pointers are host memory (memory=MEM_HOST) or device memory of the server's device
        (MEM_DEVICE); pitches in bytes (0: packed rows)."""
        req = bf_request(d, in_ptr, in_pitch or width * 4, out_ptr, out_pitch or width * 4, height, width, memory)
        t = C.c_uint64()
        _check(lib().bf_serve_submit(self._h, C.byref(req), C.byref(t)), "bf_serve_submit")
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        r = bf_result()
        st = lib().bf_serve_poll(self._h, ticket, timeout_ms, C.byref(r))
        return st, r

    def cancel(self, ticket: int) -> int:
        return lib().bf_serve_cancel(self._h, ticket)

    def close(self):
        if getattr(self, "_h", None):
            lib().bf_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
