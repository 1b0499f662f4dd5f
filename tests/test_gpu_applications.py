"""GPU parity of the paper's four applications (Figs. 1-4), each at the parameters its figure gives, s = 4.

  edge-preserving smoothing (Fig. 1)  colour image filtered with itself as guide, r = 4,  eps = 0.2^2
  detail enhancement (Fig. 2)         the same at r = 16, eps = 0.1^2, output q + 5 (I - q)
  flash / no-flash denoising (Fig. 3) clean colour image guides its noisy version, r = 8, eps = 0.02^2
  guided feathering (Fig. 4)          gray image guides a coarse binary mask, r = 60 (r' = 15), eps = 0.001^2

Colour images use one guide channel per channel of p (depthwise), the reading of the paper's colour
examples this path supports.  Inputs are synthetic stand-ins (``synth``): colour scenes, a noisy copy
(N(0, 0.1^2), clipped) and a blocky ellipse mask.  Each case runs through ``gf_filter`` at 480 x 640 against
the FP64 oracle on every pixel, and at 12 MP (4000 x 3000) on sampled bands of rows.

Tolerance: q within TOL_F32; the detail-enhanced output q + k (I - q) moves by |1 - k| times the error
of q, so it is held to |1 - k| * TOL_F32 (4e-4 at k = 5).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import TOL_F32, max_abs, oracle_q, oracle_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _inputs(app, H, W):
    """(I, p, r, eps, gain) of an application on an H x W synthetic image."""
    if app == "smoothing":
        I = synth.make_color_scene(H, W, seed=5)
        return I, I, 4, 0.2 ** 2, 0.0
    if app == "detail":
        I = synth.make_color_scene(H, W, seed=6)
        return I, I, 16, 0.1 ** 2, 5.0
    if app == "flash":
        I = synth.make_color_scene(H, W, seed=7)
        rng = np.random.default_rng(8)
        p = np.clip(I + rng.normal(0.0, 0.1, I.shape), 0.0, 1.0).astype(np.float32)
        return I, p, 8, 0.02 ** 2, 0.0
    I = synth.make_scene(H, W, seed=9)
    return I[None], synth.feather_mask(H, W, seed=10)[None], 60, 0.001 ** 2, 0.0


APPS = ["smoothing", "detail", "flash", "feathering"]


def _gpu(gf, I, p, r, eps, gain):
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, 4, "bilinear",
                              detail_gain=gain)
    torch.cuda.synchronize()
    return q.cpu().numpy()


@pytest.mark.parametrize("app", APPS)
def test_application_full_image(gf, app):
    I, p, r, eps, gain = _inputs(app, 480, 640)
    got = _gpu(gf, I, p, r, eps, gain)
    ref = oracle_q(I, p, r, eps, 4, oracle.SUB_BILINEAR)
    if gain:
        ref = oracle.detail_enhance(I.astype(np.float64), ref, gain)
    err = max_abs(got, ref)
    assert err <= max(1.0, abs(1.0 - gain)) * TOL_F32, "max-abs error %.3g" % err


@pytest.mark.parametrize("app", APPS)
def test_application_12mp_sampled_rows(gf, app):
    H, W = 3000, 4000
    I, p, r, eps, gain = _inputs(app, H, W)
    got = _gpu(gf, I, p, r, eps, gain)
    for Y0 in (0, 1498, 2990):  # top border, middle, bottom border
        Y1 = min(H, Y0 + 10)
        ref = oracle_rows(I[None], p[None], Y0, Y1, r, eps, 4, oracle.SUB_BILINEAR)[0]
        if gain:
            ref = oracle.detail_enhance(I[:, Y0:Y1].astype(np.float64), ref, gain)
        err = max_abs(got[:, Y0:Y1], ref)
        assert err <= max(1.0, abs(1.0 - gain)) * TOL_F32, "rows %d..%d: max-abs error %.3g" % (Y0, Y1, err)


def test_detail_gain_zero_and_one(gf):
    I, p, r, eps, _ = _inputs("detail", 96, 128)
    It, pt = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    q = gf.fast_guided_filter(It, pt, r, eps, 4, "bilinear")
    q0 = gf.fast_guided_filter(It, pt, r, eps, 4, "bilinear", detail_gain=0.0)
    q1 = gf.fast_guided_filter(It, pt, r, eps, 4, "bilinear", detail_gain=1.0)
    torch.cuda.synchronize()
    assert torch.equal(q, q0)
    assert float((q1 - It).abs().max()) <= 1e-6  # base layer plus the whole detail layer is the guide


def test_detail_gain_is_forward_only(gf):
    import ctypes
    I = torch.rand(1, 1, 32, 32, device="cuda")
    g = torch.empty_like(I)
    o = gf.binding.opts_init()
    o.detail_gain = 2.0
    ctx = gf.binding.default_context(I.device.index)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    st = gf.load_library().gf_filter_backward(ctx.handle, ptr(I), ptr(I), ptr(I), ptr(g), ptr(g), None, 32, 32, 1,
                                              4, 1e-2, 4, gf.GF_SUB_BILINEAR, ctypes.byref(o), None)
    assert st == gf.GF_EINVAL


@pytest.mark.parametrize("s,mode,dtype", [(4, "bilinear", torch.float32), (2, "nearest", torch.float32),
                                          (8, "box", torch.float16), (4, "bilinear", torch.uint8),
                                          (1, "bilinear", torch.float32)])
def test_self_guided_call_equals_separate_copy(gf, s, mode, dtype):
    """p passed as the guide tensor itself (subsampled once, I' reused as p') gives exactly the result of
    passing a separate copy of it."""
    I = torch.from_numpy(synth.make_color_scene(200, 328, seed=11)).cuda()
    if dtype == torch.uint8:
        I = (I * 255.0).round().to(torch.uint8)
    else:
        I = I.to(dtype)
    q_same = gf.fast_guided_filter(I, I, 8, 1e-2, s, mode)
    q_copy = gf.fast_guided_filter(I, I.clone(), 8, 1e-2, s, mode)
    torch.cuda.synchronize()
    assert torch.equal(q_same, q_copy)
