"""Helpers shared by the GPU parity tests: oracle evaluation on full images or row bands, and tolerances."""
import numpy as np

import oracle

# Max-abs tolerances of the GPU path against the FP64 oracle on [0, 1] data.
TOL_F32 = 1e-4   # FP32 storage and arithmetic
TOL_F16 = 2e-3   # FP16 storage of I, p and q, FP32 arithmetic


def oracle_q(I, p, r, eps, s, mode, r_low=None, p_lowres=False):
    return oracle.fast_guided_filter(np.asarray(I, np.float64), np.asarray(p, np.float64), r, eps, s, mode,
                                     r_low=r_low, p_lowres=p_lowres)


def oracle_rows(I, p, Y0, Y1, r, eps, s, mode):
    """Exact oracle output rows [Y0, Y1) of an (N, CI, H, W) / (N, C, H, W) problem, computed on a crop of
    full-width rows.  Output row Y depends on input rows within s * (2 r' + 3) of it, so a crop with that
    margin (started on a multiple of s so the low-res grid is the global one) reproduces those rows
    exactly, including the image's true borders where the crop touches them."""
    H = I.shape[-2]
    rl = oracle.lowres_radius(r, s)
    m = s * (2 * rl + 3) + s
    ys = max(0, Y0 - m) // s * s
    ye = min(H, Y1 + m)
    q = oracle.fast_guided_filter(np.asarray(I[..., ys:ye, :], np.float64), np.asarray(p[..., ys:ye, :], np.float64),
                                  r, eps, s, mode, r_low=rl)
    return q[..., Y0 - ys:Y1 - ys, :]


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))))
