"""ctypes binding of libgf.so: the names of include/gf.h, with torch tensors for device memory and streams.

This module only marshals arguments; every step of the filter runs in the library's CUDA kernels.  If the
library cannot be loaded the calls raise -- there is no CPU fallback.
"""
import ctypes
import math
import os
import threading
from fractions import Fraction

import torch

from . import _build

GF_OK, GF_PENDING, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ETIMEOUT, GF_EBUSY, GF_ECANCELED, GF_ENOTFOUND, GF_EWAIT = \
    0, 1, -1, -2, -3, -4, -5, -6, -7, -8
GF_SUB_NEAREST, GF_SUB_BILINEAR, GF_SUB_BOX, GF_SUB_BILINEAR_AA = 0, 1, 2, 3
GF_F32, GF_F16, GF_U8 = 0, 1, 2
GF_MAX_STAGES = 8

MODES = {"nearest": GF_SUB_NEAREST, "bilinear": GF_SUB_BILINEAR, "box": GF_SUB_BOX,
         "bilinear_aa": GF_SUB_BILINEAR_AA}
_DTYPES = {torch.float32: GF_F32, torch.float16: GF_F16, torch.uint8: GF_U8}
_STATUS_NAMES = {0: "GF_OK", 1: "GF_PENDING", -1: "GF_EINVAL", -2: "GF_ENOMEM", -3: "GF_ECUDA",
                 -4: "GF_ETIMEOUT", -5: "GF_EBUSY", -6: "GF_ECANCELED", -7: "GF_ENOTFOUND", -8: "GF_EWAIT"}


class GFError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), message))
        self.status = status


ABI_VERSION = 5  # GF_ABI_VERSION of include/gf.h that GFOpts mirrors


class GFOpts(ctypes.Structure):
    _fields_ = [
        ("batch", ctypes.c_int),
        ("guide_channels", ctypes.c_int),
        ("r_low", ctypes.c_int),
        ("p_lowres", ctypes.c_int),
        ("dtype_in", ctypes.c_int),
        ("dtype_out", ctypes.c_int),
        ("a_out", ctypes.c_void_p),
        ("b_out", ctypes.c_void_p),
        ("mean_a_out", ctypes.c_void_p),
        ("mean_b_out", ctypes.c_void_p),
        ("stats_out", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("kernel_events", ctypes.c_void_p),
        ("detail_gain", ctypes.c_float),
        ("row_begin", ctypes.c_int),
        ("row_end", ctypes.c_int),
        ("color_guide", ctypes.c_int),
        ("s_num", ctypes.c_int),
        ("s_den", ctypes.c_int),
        ("fused", ctypes.c_int),
        ("saved_forward", ctypes.c_int),
        ("test_wait_fault", ctypes.c_int),
    ]


class GFRequest(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_void_p), ("p", ctypes.c_void_p), ("q", ctypes.c_void_p),
        ("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int), ("r", ctypes.c_int),
        ("eps", ctypes.c_float), ("s", ctypes.c_int), ("mode", ctypes.c_int),
        ("opts", GFOpts), ("user", ctypes.c_void_p), ("ready_event", ctypes.c_void_p),
    ]


class GFResult(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("ticket", ctypes.c_uint64), ("user", ctypes.c_void_p),
        ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
        ("scratch_bytes", ctypes.c_size_t),
    ]


class GFServeStats(ctypes.Structure):
    _fields_ = [
        ("queued", ctypes.c_int), ("running", ctypes.c_int), ("slots", ctypes.c_int),
        ("budget_bytes", ctypes.c_size_t), ("scratch_in_use", ctypes.c_size_t),
        ("launches", ctypes.c_longlong), ("graph_launches", ctypes.c_longlong),
        ("queue_launches", ctypes.c_longlong), ("queue_requests", ctypes.c_longlong), ("launch_seconds", ctypes.c_double),
    ]


_lib = None
_lib_lock = threading.Lock()


def library_path():
    return _build.LIB_PATH


def load_library(build_if_missing=True):
    """Load libgf.so (building it first if it is missing and ``build_if_missing``).  Raises if it cannot
    be loaded: callers never fall back to another implementation."""
    global _lib
    if _lib is not None:  # loaded: no lock on the per-call path
        return _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing and _build.needs_build():
            _build.build_library()
        if not os.path.exists(path):
            raise RuntimeError("libgf.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        vp, i, f, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
        P = ctypes.POINTER
        lib.gf_opts_init.argtypes = [P(GFOpts)]
        lib.gf_opts_init.restype = None
        lib.gf_abi_version.restype = i
        if lib.gf_abi_version() != ABI_VERSION:
            raise RuntimeError("libgf.so has ABI version %d, this binding needs %d: rebuild it"
                               % (lib.gf_abi_version(), ABI_VERSION))
        lib.gf_last_error.restype = ctypes.c_char_p
        lib.gf_lowres_geometry.argtypes = [i, i, i, i, i, P(i), P(i), P(i)]
        lib.gf_lowres_geometry.restype = i
        lib.gf_workspace_size.argtypes = [i, i, i, i, P(GFOpts), P(sz)]
        lib.gf_workspace_size.restype = i
        lib.gf_kernel_faults.argtypes = [i, P(ctypes.c_uint), i]
        lib.gf_kernel_faults.restype = i
        lib.gf_row_band.argtypes = [i, i, i, i, i, i, i, i, P(i), P(i)]
        lib.gf_row_band.restype = i
        lib.gf_filter_kernel_count.argtypes = [i, i, i, i, i, P(GFOpts)]
        lib.gf_filter_kernel_count.restype = i
        lib.gf_create.argtypes = [P(vp), i, sz, ctypes.c_uint]
        lib.gf_create.restype = i
        lib.gf_destroy.argtypes = [vp]
        lib.gf_destroy.restype = i
        lib.gf_filter.argtypes = [vp, vp, vp, vp, i, i, i, i, f, i, i, P(GFOpts), vp]
        lib.gf_filter.restype = i
        lib.gf_filter_host.argtypes = [vp, vp, vp, vp, i, i, i, i, f, i, i, P(GFOpts), vp]
        lib.gf_filter_host.restype = i
        lib.gf_host_strips.argtypes = [i, i, i, i, i, P(GFOpts), P(i)]
        lib.gf_host_strips.restype = i
        lib.gf_filter_noalloc.argtypes = [vp, vp, vp, i, i, i, i, f, i, i, P(GFOpts), vp]
        lib.gf_filter_noalloc.restype = i
        lib.gf_backward_workspace_size.argtypes = [i, i, i, i, P(GFOpts), P(sz)]
        lib.gf_backward_workspace_size.restype = i
        lib.gf_filter_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, i, i, i, f, i, i, P(GFOpts), vp]
        lib.gf_filter_backward.restype = i
        lib.gf_clock.restype = ctypes.c_double
        lib.gf_serve_config.argtypes = [vp, i, sz]
        lib.gf_serve_config.restype = i
        lib.gf_serve_pause.argtypes = [vp, i]
        lib.gf_serve_pause.restype = i
        lib.gf_serve_graphs.argtypes = [vp, i]
        lib.gf_serve_graphs.restype = i
        lib.gf_serve_tile_queue.argtypes = [vp, i]
        lib.gf_serve_tile_queue.restype = i
        lib.gf_submit.argtypes = [vp, P(GFRequest), P(ctypes.c_uint64)]
        lib.gf_submit.restype = i
        lib.gf_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64, P(GFResult)]
        lib.gf_poll.restype = i
        lib.gf_cancel.argtypes = [vp, ctypes.c_uint64]
        lib.gf_cancel.restype = i
        lib.gf_serve_stats_get.argtypes = [vp, P(GFServeStats)]
        lib.gf_serve_stats_get.restype = i
        _lib = lib
        return lib


def check(status):
    if status != GF_OK:
        msg = load_library(False).gf_last_error().decode(errors="replace")
        raise GFError(status, msg)
    return status


_DEFAULT_OPTS = None  # gf_opts_init's result, copied for every call


def opts_init():
    global _DEFAULT_OPTS
    if _DEFAULT_OPTS is None:
        o = GFOpts()
        load_library().gf_opts_init(ctypes.byref(o))
        _DEFAULT_OPTS = bytes(o)
    return GFOpts.from_buffer_copy(_DEFAULT_OPTS)


def kernel_faults(device=None, clear=True):
    """Fault bits the kernels recorded on `device` since the last clear (bit 0: a bounded wait of the TMA output
    kernel gave up, bit 1: of a TMA box kernel); cleared by default."""
    if device is None:
        device = torch.cuda.current_device()
    v = ctypes.c_uint()
    check(load_library().gf_kernel_faults(int(device), ctypes.byref(v), int(bool(clear))))
    return v.value


def _integer_ratio(s):
    f = Fraction(s)
    if f.denominator != 1:
        raise ValueError("this call takes an integer ratio s")
    return int(f)


def lowres_geometry(H, W, s, r, r_low=-1):
    h, w, rp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(load_library().gf_lowres_geometry(int(H), int(W), _integer_ratio(s), int(r), int(r_low), ctypes.byref(h),
                                            ctypes.byref(w), ctypes.byref(rp)))
    return h.value, w.value, rp.value


def _ratio(o, s):
    """The integer s to pass with options `o`: an integer ratio as it is; a non-integer one (a Fraction, or
    a float that is an exact binary fraction such as 2.5) goes into o.s_num / o.s_den."""
    if type(s) is int:
        return s
    f = Fraction(s)
    if f.denominator == 1:
        return int(f)
    o.s_num, o.s_den = f.numerator, f.denominator
    return math.ceil(f)


def row_band(H, W, s, r, row_begin, row_end, r_low=-1, mode="bilinear"):
    """(row0, rows): the full-res input rows a call restricted to output rows [row_begin, row_end) reads."""
    a, b = ctypes.c_int(), ctypes.c_int()
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    check(load_library().gf_row_band(int(H), int(W), _integer_ratio(s), int(r), int(r_low), m, int(row_begin),
                                     int(row_end), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def host_strips(H, W, C, s, mode="bilinear", *, batch=1, guide_channels=1, dtype=torch.float32, out_dtype=None):
    """Row boundaries [0, ..., H] of the strips ``gf_filter_host`` pipelines such a call in, or None when it
    copies in, filters and copies out in one piece."""
    o = opts_init()
    o.batch = int(batch)
    o.guide_channels = int(guide_channels)
    s = _ratio(o, s)
    o.dtype_in = _DTYPES[dtype]
    o.dtype_out = _DTYPES[out_dtype or (torch.float16 if dtype == torch.float16 else torch.float32)]
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    ys = (ctypes.c_int * 9)()  # gf_host_strips writes at most 9 boundaries
    k = load_library().gf_host_strips(int(H), int(W), int(C), int(s), m, ctypes.byref(o), ys)
    if k < 0:
        check(GF_EINVAL)
    return list(ys[:k + 1]) if k >= 2 else None


def row_strips(H, parts, align=1):
    """Split rows [0, H) into `parts` contiguous strips of nearly equal height whose inner boundaries are
    multiples of `align` (one strip per device of a row-sharded filter).  Returns [(row_begin, row_end)]."""
    if parts < 1 or H < 1:
        raise ValueError("parts and H must be >= 1")
    cuts = [0]
    for k in range(1, parts):
        cuts.append(min(H, max(cuts[-1], int(round(k * H / parts / align)) * align)))
    cuts.append(H)
    return [(cuts[k], cuts[k + 1]) for k in range(parts)]


class Context:
    """Owns a gf_ctx (scratch arena, serving state) on one CUDA device."""

    def __init__(self, device=None, hbm_budget_bytes=0):
        lib = load_library()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        self._ptr = ctypes.c_void_p()
        check(lib.gf_create(ctypes.byref(self._ptr), self.device, int(hbm_budget_bytes), 0))

    @property
    def handle(self):
        return self._ptr

    def close(self):
        if self._ptr:
            check(load_library().gf_destroy(self._ptr))
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts = {}


def default_context(device=None):
    if device is None:
        device = torch.cuda.current_device()
    device = int(device)
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


def _nchw(x, name):
    if x.dim() == 2:
        return x[None, None], 2
    if x.dim() == 3:
        return x[None], 3
    if x.dim() == 4:
        return x, 4
    raise ValueError("%s must have 2, 3 or 4 dimensions" % name)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def fast_guided_filter(I, p, r, eps, s=4, mode="bilinear", *, r_low=None, p_lowres=False, out_dtype=None,
                       out=None, a_out=None, b_out=None, mean_a_out=None, mean_b_out=None, stats_out=None,
                       workspace=None, kernel_events=None, stream=None, ctx=None, detail_gain=0.0, rows=None,
                       color_guide=False, fused=0, saved_forward=False, test_wait_fault=False):
    """Fast guided filter (Algorithm 2; Algorithm 1 at s = 1) on CUDA tensors, via ``gf_filter``.

    I: (H, W), (CI, H, W) or (N, CI, H, W); p: the same rank with C channels (at low resolution when
    ``p_lowres``).  CI is 1 or C.  dtypes: float32, float16 or uint8 (I and p alike).  Returns q shaped like
    p at full resolution, float32 (float16 for float16 input unless ``out_dtype`` says otherwise).
    ``detail_gain`` k != 0 returns q + k (I - q) instead (detail enhancement when p is I).
    ``rows=(row_begin, row_end)`` computes only those output rows of q (needs ``out``, the whole q, whose
    other rows are left as they are): one strip of an image split across devices or streams.
    ``color_guide=True``: I has 3 channels used jointly as a colour guide for every channel of p.
    ``fused``: 0 runs the whole filter as one kernel for small images, 1 always, -1 never.
    ``saved_forward=True`` with ``workspace`` (``backward_workspace_size`` bytes) keeps the low-res planes
    there for a ``fast_guided_filter_backward`` call with the same arguments, workspace and flag.
    ``test_wait_fault=True`` is the test hook of gf_opts.test_wait_fault (a bounded wait is made to run out).
    """
    if not (I.is_cuda and p.is_cuda):
        raise ValueError("I and p must be CUDA tensors")
    if I.dtype != p.dtype or I.dtype not in _DTYPES:
        raise ValueError("I and p must share one of float32, float16, uint8")
    I4, _ = _nchw(I, "I")
    p4, prank = _nchw(p, "p")
    N, CI, H, W = I4.shape
    C = p4.shape[1]
    if p4.shape[0] != N:
        raise ValueError("I and p must have the same batch size")
    if out_dtype is None:
        out_dtype = torch.float16 if I.dtype == torch.float16 else torch.float32
    if out_dtype not in (torch.float32, torch.float16):
        raise ValueError("out_dtype must be float32 or float16")
    qshape = (N, C, H, W)
    given = out is not None
    if out is None:
        out = torch.empty(qshape, dtype=out_dtype, device=I.device)
    elif out.numel() != N * C * H * W or out.dtype != out_dtype or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous CUDA %s tensor of %d elements" % (out_dtype, N * C * H * W))
    result = out
    out = out.view(qshape)
    if min(N, C, H, W) == 0 or p4.numel() == 0:
        return result if given else (out.reshape(p.shape[:-2] + (H, W)) if prank < 4 else out)
    I4 = I4.contiguous()
    p4 = p4.contiguous()
    o = opts_init()
    o.batch = N
    o.guide_channels = CI
    o.r_low = -1 if r_low is None else int(r_low)
    s = _ratio(o, s)
    o.p_lowres = int(bool(p_lowres))
    o.dtype_in = _DTYPES[I.dtype]
    o.dtype_out = _DTYPES[out_dtype]
    o.detail_gain = float(detail_gain)
    o.color_guide = int(bool(color_guide))
    o.fused = int(fused)
    o.saved_forward = int(bool(saved_forward))
    o.test_wait_fault = int(bool(test_wait_fault))
    if rows is not None:
        if not given:
            raise ValueError("rows needs out= (the whole q; rows outside the range are not written)")
        o.row_begin, o.row_end = int(rows[0]), int(rows[1])
    for name, t in (("a_out", a_out), ("b_out", b_out), ("mean_a_out", mean_a_out),
                    ("mean_b_out", mean_b_out), ("stats_out", stats_out)):
        if t is not None:
            if not t.is_contiguous():
                raise ValueError("%s must be contiguous" % name)
            setattr(o, name, t.data_ptr())
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    ev_arr = None
    if kernel_events is not None:
        if len(kernel_events) != 2 * GF_MAX_STAGES:
            raise ValueError("kernel_events needs %d events" % (2 * GF_MAX_STAGES))
        st = stream if stream is not None else torch.cuda.current_stream()
        for e in kernel_events:
            if not e.cuda_event:  # torch creates the CUDA event on its first record
                e.record(st)
        ev_arr = (ctypes.c_void_p * (2 * GF_MAX_STAGES))(*[e.cuda_event for e in kernel_events])
        o.kernel_events = ctypes.cast(ev_arr, ctypes.c_void_p)
    dev = I.device.index
    ctx = ctx or default_context(dev)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if stream is None:
        stream = torch.cuda.current_stream(dev)  # the current stream of I's device; the library sets the device
    check(load_library().gf_filter(ctx.handle, _ptr(I4), _ptr(p4), _ptr(out), H, W, C, int(r), float(eps),
                                   int(s), m, ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream)))
    if given:
        return result
    if prank == 2:
        return out[0, 0]
    if prank == 3:
        return out[0]
    return out


def fast_guided_filter_host(I, p, r, eps, s=4, mode="bilinear", *, out=None, out_dtype=None, r_low=None,
                            stream=None, ctx=None, device=None, fused=0, test_wait_fault=False):
    """Same filter on HOST (CPU) tensors through ``gf_filter_host``: the library copies the inputs to the
    device, filters and copies q back before returning.  A kernel that gave up a bounded wait makes it raise
    GFError with status GF_EWAIT."""
    if I.is_cuda or p.is_cuda:
        raise ValueError("gf_filter_host takes host tensors")
    I4, _ = _nchw(I, "I")
    p4, prank = _nchw(p, "p")
    N, CI, H, W = I4.shape
    C = p4.shape[1]
    if out_dtype is None:
        out_dtype = torch.float16 if I.dtype == torch.float16 else torch.float32
    if out is None:
        out = torch.empty((N, C, H, W), dtype=out_dtype)
    o = opts_init()
    o.batch = N
    o.guide_channels = CI
    o.r_low = -1 if r_low is None else int(r_low)
    s = _ratio(o, s)
    o.dtype_in = _DTYPES[I.dtype]
    o.dtype_out = _DTYPES[out_dtype]
    o.fused = int(fused)
    o.test_wait_fault = int(bool(test_wait_fault))
    ctx = ctx or default_context(device)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    I4 = I4.contiguous()
    p4 = p4.contiguous()
    with torch.cuda.device(ctx.device):
        check(load_library().gf_filter_host(ctx.handle, _ptr(I4), _ptr(p4), _ptr(out), H, W, C, int(r),
                                            float(eps), int(s), m, ctypes.byref(o), _stream_handle(stream)))
    return out.reshape(p.shape[:-2] + (H, W)) if prank < 4 else out


def backward_workspace_size(H, W, C, s=4, *, batch=1, guide_channels=1, r_low=None, p_lowres=False):
    """Bytes of scratch a backward call (and a forward call that saves for it) needs."""
    o = opts_init()
    o.batch, o.guide_channels = int(batch), int(guide_channels)
    o.r_low = -1 if r_low is None else int(r_low)
    o.p_lowres = int(bool(p_lowres))
    s = _ratio(o, s)
    n = ctypes.c_size_t()
    check(load_library().gf_backward_workspace_size(int(H), int(W), int(C), int(s), ctypes.byref(o), ctypes.byref(n)))
    return n.value


def fast_guided_filter_backward(I, p, dq, r, eps, s=4, mode="bilinear", *, r_low=None, p_lowres=False,
                                need_eps=True, stream=None, ctx=None, workspace=None, saved_forward=False):
    """Backward pass of ``fast_guided_filter`` via ``gf_filter_backward`` (FP32 CUDA tensors).

    dq has the shape of q.  Returns (dI, dp, deps): dI shaped like I, dp shaped like p, deps a 0-dim
    device tensor (or None when ``need_eps`` is False).  ``workspace``: optional scratch of
    ``backward_workspace_size`` bytes; with ``saved_forward=True`` it holds the low-res planes a
    ``fast_guided_filter(..., saved_forward=True)`` call with the same arguments left there, and they are
    not recomputed."""
    if not (I.is_cuda and p.is_cuda and dq.is_cuda):
        raise ValueError("I, p and dq must be CUDA tensors")
    if I.dtype != torch.float32 or p.dtype != torch.float32 or dq.dtype != torch.float32:
        raise ValueError("the backward pass takes float32 tensors")
    I4, irank = _nchw(I, "I")
    p4, prank = _nchw(p, "p")
    N, CI, H, W = I4.shape
    C = p4.shape[1]
    dq4 = dq.reshape(N, C, H, W).contiguous()
    I4 = I4.contiguous()
    p4 = p4.contiguous()
    dI = torch.empty_like(I4)
    dp = torch.empty_like(p4)
    deps = torch.empty((), dtype=torch.float32, device=I.device) if need_eps else None
    o = opts_init()
    o.batch = N
    o.guide_channels = CI
    o.r_low = -1 if r_low is None else int(r_low)
    s = _ratio(o, s)
    o.p_lowres = int(bool(p_lowres))
    o.saved_forward = int(bool(saved_forward))
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    ctx = ctx or default_context(I.device.index)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    with torch.cuda.device(I.device):
        check(load_library().gf_filter_backward(ctx.handle, _ptr(I4), _ptr(p4), _ptr(dq4), _ptr(dI), _ptr(dp),
                                                _ptr(deps), H, W, C, int(r), float(eps), int(s), m, ctypes.byref(o),
                                                _stream_handle(stream)))
    return dI.reshape(I.shape), dp.reshape(p.shape), deps
