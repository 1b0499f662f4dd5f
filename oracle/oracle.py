"""ctypes front end of the FP64 C oracle (``gf_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the benchmark's CPU-baseline leg.
Every function takes and returns float64 numpy arrays; the C side does all of the arithmetic.
"""
import contextlib
import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

SUB_NEAREST, SUB_BILINEAR, SUB_BOX, SUB_BILINEAR_AA = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgforacle.so")
_lock = threading.Lock()
_lib = None


def compile_library(src, out):
    """gcc ``src`` (a copy of ``gf_oracle.c``) into the shared library ``out`` with the oracle's flags (no FMA
    contraction, so that x86 and Arm hosts round the same way)."""
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, src, "-lm"])


def build(force=False):
    """Compile ``gf_oracle.c`` with gcc into ``oracle/_build/libgforacle.so`` (no FMA contraction, so that
    x86 and Arm hosts round the same way).  Returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        compile_library(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declare the argument types of the C entry points on a loaded build of ``gf_oracle.c``."""
    D = ctypes.POINTER(ctypes.c_double)
    i, d = ctypes.c_int, ctypes.c_double
    lib.gfo_lowres_radius.argtypes = [i, i]
    lib.gfo_lowres_radius.restype = i
    lib.gfo_lowres_shape.argtypes = [i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.gfo_lowres_radius_q.argtypes = [i, i, i]
    lib.gfo_lowres_radius_q.restype = i
    lib.gfo_lowres_shape_q.argtypes = [i, i, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.gfo_subsample_q.argtypes = [D, i, i, i, i, i, D]
    lib.gfo_upsample_q.argtypes = [D, i, i, i, i, i, i, D]
    lib.gfo_fast_guided_filter_q.argtypes = [D, D, i, i, i, i, i, i, d, i, i, i, i, i, D, D, D, D, D, D]
    lib.gfo_fast_guided_filter_q.restype = i
    lib.gfo_subsample.argtypes = [D, i, i, i, i, D]
    for name in ("gfo_box_sum", "gfo_box_mean", "gfo_box_mean_bruteforce"):
        getattr(lib, name).argtypes = [D, i, i, i, D]
    lib.gfo_upsample.argtypes = [D, i, i, i, i, i, D]
    lib.gfo_fast_guided_filter.argtypes = [D, D, i, i, i, i, i, i, d, i, i, i, i, D, D, D, D, D, D]
    lib.gfo_fast_guided_filter.restype = i
    lib.gfo_guided_filter.argtypes = [D, D, i, i, i, d, D]
    lib.gfo_guided_filter.restype = i
    lib.gfo_fast_guided_filter_backward.argtypes = [D, D, D, i, i, i, i, i, i, d, i, i, i, i, D, D, D]
    lib.gfo_fast_guided_filter_backward.restype = i
    lib.gfo_color_guided_filter.argtypes = [D, D, i, i, i, i, i, d, i, i, i, D, D, D]
    lib.gfo_color_guided_filter.restype = i
    lib.gfo_detail_enhance.argtypes = [D, D, i, i, i, i, i, d, D]
    lib.gfo_detail_enhance.restype = i
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def use_library(path):
    """Run every oracle function from another build of ``gf_oracle.c`` (the shared library at ``path``)
    while the block runs; the mutation tests use it to run the pins on copies with a planted mistake."""
    global _lib
    _load()
    variant = _bind(ctypes.CDLL(path))
    with _lock:
        saved, _lib = _lib, variant
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _c64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(x):
    if x is None:
        return None
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ratio(s):
    """The subsampling ratio as (sn, sd) with s = sn / sd: an int, a fractions.Fraction, or a float that is
    an exact binary fraction (e.g. 2.5)."""
    f = Fraction(s)
    if f < 1:
        raise ValueError("the ratio s must be >= 1")
    return f.numerator, f.denominator


def lowres_radius(r, s):
    """r' = r/s rounded half up, at least 1 when r >= 1; s = 1 gives r."""
    sn, sd = ratio(s)
    return int(_load().gfo_lowres_radius_q(int(r), sn, sd))


def lowres_shape(H, W, s):
    sn, sd = ratio(s)
    h, w = ctypes.c_int(), ctypes.c_int()
    _load().gfo_lowres_shape_q(int(H), int(W), sn, sd, ctypes.byref(h), ctypes.byref(w))
    return h.value, w.value


def subsample(x, s, mode):
    x = _c64(x)
    H, W = x.shape
    h, w = lowres_shape(H, W, s)
    y = np.empty((h, w), np.float64)
    sn, sd = ratio(s)
    if mode == SUB_BOX and sd != 1:
        raise ValueError("box subsampling needs an integer ratio")
    _load().gfo_subsample_q(_ptr(x), H, W, sn, sd, int(mode), _ptr(y))
    return y


def _box(name, x, r):
    x = _c64(x)
    h, w = x.shape
    y = np.empty_like(x)
    getattr(_load(), name)(_ptr(x), h, w, int(r), _ptr(y))
    return y


def box_sum(x, r):
    return _box("gfo_box_sum", x, r)


def box_mean(x, r):
    return _box("gfo_box_mean", x, r)


def box_mean_bruteforce(x, r):
    return _box("gfo_box_mean_bruteforce", x, r)


def upsample(x, s, H, W):
    x = _c64(x)
    h, w = x.shape
    y = np.empty((H, W), np.float64)
    sn, sd = ratio(s)
    _load().gfo_upsample_q(_ptr(x), h, w, sn, sd, int(H), int(W), _ptr(y))
    return y


def _as_nchw(x):
    x = _c64(x)
    if x.ndim == 2:
        return x[None, None], 2
    if x.ndim == 3:
        return x[None], 3
    return x, 4


def fast_guided_filter(I, p, r, eps, s, mode=SUB_BILINEAR, r_low=None, p_lowres=False, brute=False,
                       intermediates=False):
    """Algorithm 2 in FP64.

    I: (H, W), (CI, H, W) or (N, CI, H, W); p: same rank with C channels (at h x w when ``p_lowres``).
    r is the full-res radius; ``r_low`` overrides r' (else r' = lowres_radius(r, s)).
    Returns q shaped like p at full resolution, plus a dict of low-res intermediates when asked
    (``a``, ``b``, ``mean_a``, ``mean_b``: N x C x h x w; ``stats``: N x C x 4 x h x w with
    mean_I, corr_I, mean_p, corr_Ip).
    """
    I4, _ = _as_nchw(I)
    p4, prank = _as_nchw(p)
    N, CI, H, W = I4.shape
    C = p4.shape[1]
    if p4.shape[0] != N:
        raise ValueError("batch mismatch")
    h, w = lowres_shape(H, W, s)
    rl = lowres_radius(r, s) if r_low is None else int(r_low)
    q = np.empty((N, C, H, W), np.float64)
    inter = None
    if intermediates:
        inter = {k: np.empty((N, C, h, w), np.float64) for k in ("a", "b", "mean_a", "mean_b")}
        inter["stats"] = np.empty((N, C, 4, h, w), np.float64)
    g = (lambda k: _ptr(inter[k])) if inter else (lambda k: None)
    sn, sd = ratio(s)
    rc = _load().gfo_fast_guided_filter_q(_ptr(I4), _ptr(p4), N, CI, C, H, W, rl, float(eps), sn, sd, int(mode),
                                        int(bool(p_lowres)), int(bool(brute)), _ptr(q), g("a"), g("b"),
                                        g("mean_a"), g("mean_b"), g("stats"))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    if prank == 2:
        q = q[0, 0]
        if inter:
            inter = {k: v[0, 0] for k, v in inter.items()}
    elif prank == 3:
        q = q[0]
        if inter:
            inter = {k: v[0] for k, v in inter.items()}
    return (q, inter) if intermediates else q


def color_guided_filter(I, p, r, eps, s, mode=SUB_BILINEAR, r_low=None, p_lowres=False, intermediates=False):
    """Colour-guided fast guided filter (R12) in FP64.  I: (3, H, W) or (N, 3, H, W); p: (C, H, W) or
    (N, C, H, W) (at h x w when ``p_lowres``).  Returns q shaped like p at full resolution, plus
    {"a": N x C x 3 x h x w, "b": N x C x h x w} when ``intermediates``."""
    I4, _ = _as_nchw(I)
    p4, prank = _as_nchw(p)
    N, CI, H, W = I4.shape
    C = p4.shape[1]
    if CI != 3 or p4.shape[0] != N:
        raise ValueError("the colour guide has 3 channels and the batch sizes must match")
    h, w = lowres_shape(H, W, s)
    rl = lowres_radius(r, s) if r_low is None else int(r_low)
    q = np.empty((N, C, H, W), np.float64)
    a = np.empty((N, C, 3, h, w), np.float64) if intermediates else None
    b = np.empty((N, C, h, w), np.float64) if intermediates else None
    rc = _load().gfo_color_guided_filter(_ptr(I4), _ptr(p4), N, C, H, W, rl, float(eps), int(s), int(mode),
                                         int(bool(p_lowres)), _ptr(q), _ptr(a) if intermediates else None,
                                         _ptr(b) if intermediates else None)
    if rc != 0:
        raise ValueError("oracle rejected the arguments" if rc == -1 else "singular Sigma + eps U")
    if prank == 3:
        q = q[0]
    return (q, {"a": a, "b": b}) if intermediates else q


def detail_enhance(I, q, k):
    """q + k (I - q) (Fig. 2's detail enhancement; I is the guide, one channel shared or one per channel).
    I: (N, CI, H, W) or lower rank like q; returns an array shaped like q."""
    I4, _ = _as_nchw(I)
    q4, qrank = _as_nchw(q)
    N, CI, H, W = I4.shape
    C = q4.shape[1]
    out = np.empty_like(q4)
    if _load().gfo_detail_enhance(_ptr(I4), _ptr(q4), N, CI, C, H, W, float(k), _ptr(out)) != 0:
        raise ValueError("oracle rejected the arguments")
    return out.reshape(np.shape(q))


def guided_filter(I, p, r, eps):
    """Algorithm 1 (separately coded, summed-area-table box filter) on one plane."""
    I = _c64(I)
    p = _c64(p)
    H, W = I.shape
    q = np.empty_like(I)
    if _load().gfo_guided_filter(_ptr(I), _ptr(p), H, W, int(r), float(eps), _ptr(q)) != 0:
        raise ValueError("oracle rejected the arguments")
    return q


def fast_guided_filter_backward(I, p, gq, r, eps, s, mode=SUB_BILINEAR, r_low=None, p_lowres=False,
                                brute=False):
    """Adjoint of Algorithm 2: returns (dI, dp, deps) for the upstream gradient gq (shaped like q)."""
    I4, irank = _as_nchw(I)
    p4, prank = _as_nchw(p)
    g4, _ = _as_nchw(gq)
    N, CI, H, W = I4.shape
    C = p4.shape[1]
    rl = lowres_radius(r, s) if r_low is None else int(r_low)
    dI = np.empty_like(I4)
    dp = np.empty_like(p4)
    deps = np.zeros(1, np.float64)
    rc = _load().gfo_fast_guided_filter_backward(_ptr(I4), _ptr(p4), _ptr(g4), N, CI, C, H, W, rl, float(eps),
                                                 int(s), int(mode), int(bool(p_lowres)), int(bool(brute)),
                                                 _ptr(dI), _ptr(dp), _ptr(deps))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    shape_I = {2: lambda x: x[0, 0], 3: lambda x: x[0], 4: lambda x: x}
    return shape_I[irank](dI), shape_I[prank](dp), float(deps[0])
