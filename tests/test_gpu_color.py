"""GPU parity of the colour-guided form (gf_opts.color_guide) against the FP64 oracle.

The guide has 3 channels used jointly: per window a = (Sigma + eps U)^-1 cov_Ip with Sigma the 3 x 3
covariance of the subsampled guide, b = mean_p - a^T mean_I, q = mean_a^T I + mean_b.  Checks: every pixel
against the oracle on ragged and multi-tile shapes, every subsample mode, s = 1 .. 8, batches, one or three
channels of p, a low-res p, FP16 storage, the detail epilogue; a gray guide replicated in three channels
equals the gray path with eps / 3; a self-guided call; row strips; 12 MP guided feathering (the paper's
Fig. 4 setting: colour image, binary mask, r = 60, eps = 0.001^2, s = 4) on sampled rows.

Tolerance: TOL_F32 (TOL_F16 for FP16 storage).  The 3 x 3 solve runs in FP32 on covariances taken
relative to one sample of each plane; on these inputs (per-channel noise, so Sigma is far from singular
at the eps used) its rounding stays well inside the bound.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import TOL_F16, TOL_F32, max_abs

pytestmark = pytest.mark.gpu

MODES = {"nearest": oracle.SUB_NEAREST, "bilinear": oracle.SUB_BILINEAR, "box": oracle.SUB_BOX,
         "bilinear_aa": oracle.SUB_BILINEAR_AA}


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _inputs(N, C, H, W, seed, p_lowres=False, s=1):
    I = np.stack([synth.make_color_scene(H, W, seed=seed + k) for k in range(N)])
    rng = np.random.default_rng(seed + 100)
    if p_lowres:
        p = rng.uniform(0, 1, (N, C, -(-H // s), -(-W // s))).astype(np.float32)
    else:
        p = np.clip(I[:, :C] + rng.normal(0, 0.1, (N, C, H, W)), 0, 1).astype(np.float32) if C <= 3 else \
            rng.uniform(0, 1, (N, C, H, W)).astype(np.float32)
    return I, p


CASES = [  # (N, C, H, W, r, eps, s, mode, p_lowres)
    (1, 1, 64, 96, 8, 1e-2, 4, "bilinear", False),
    (1, 3, 120, 200, 16, 1e-3, 4, "bilinear", False),
    (2, 2, 61, 43, 6, 1e-3, 3, "nearest", False),
    (1, 3, 100, 130, 8, 1e-2, 1, "bilinear", False),
    (1, 1, 203, 408, 16, 1e-3, 8, "bilinear_aa", False),
    (2, 3, 96, 128, 0, 1e-2, 4, "box", True),
    (1, 4, 257, 1030, 24, 1e-4, 8, "bilinear", False),
    (1, 3, 136, 264, 16, 1e-3, 8, "bilinear", False),    # s = 8 run form of the output, C = 3
    (1, 3, 300, 1100, 16, 1e-3, 4, "bilinear", False),   # 3 output bands (the last 76 pixels), h = 75 ragged
    (1, 1, 7, 5, 4, 1e-2, 2, "bilinear", False),
]


def _gpu(gf, I, p, r, eps, s, mode, **kw):
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, mode,
                              color_guide=True, **kw)
    torch.cuda.synchronize()
    return q.float().cpu().numpy()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%dC%d_%dx%d_r%d_s%d_%s%s" % (
    c[0], c[1], c[2], c[3], c[4], c[6], c[7], "_plow" if c[8] else ""))
def test_color_parity(gf, case):
    N, C, H, W, r, eps, s, mode, p_lowres = case
    I, p = _inputs(N, C, H, W, seed=H + W, p_lowres=p_lowres, s=s)
    kw = {"r_low": 2, "p_lowres": True} if p_lowres else {}
    got = _gpu(gf, I, p, r, eps, s, mode, **kw)
    ref = oracle.color_guided_filter(I.astype(np.float64), p.astype(np.float64), r, eps, s, MODES[mode], **kw)
    err = max_abs(got, ref)
    assert err <= TOL_F32, "max-abs error %.3g" % err


def test_color_fp16_storage(gf):
    I, p = _inputs(1, 3, 150, 244, seed=3)
    I16, p16 = I.astype(np.float16), p.astype(np.float16)
    q = gf.fast_guided_filter(torch.from_numpy(I16).cuda(), torch.from_numpy(p16).cuda(), 8, 1e-2, 4, "bilinear",
                              color_guide=True)
    torch.cuda.synchronize()
    assert q.dtype == torch.float16
    ref = oracle.color_guided_filter(I16.astype(np.float64), p16.astype(np.float64), 8, 1e-2, 4, oracle.SUB_BILINEAR)
    assert max_abs(q.float().cpu().numpy(), ref) <= TOL_F16


def test_color_detail_epilogue(gf):
    I, _ = _inputs(1, 3, 120, 160, seed=4)
    got = _gpu(gf, I, I, 16, 0.1 ** 2, 4, "bilinear", detail_gain=5.0)
    q = oracle.color_guided_filter(I.astype(np.float64), I.astype(np.float64), 16, 0.1 ** 2, 4, oracle.SUB_BILINEAR)
    ref = oracle.detail_enhance(I.astype(np.float64), q, 5.0)
    assert max_abs(got, ref) <= 4 * TOL_F32


def test_replicated_gray_guide_equals_gray_path_with_eps_over_3(gf):
    G = synth.make_scene(300, 520, seed=6)[None, None]
    p = synth.rgb_noisy_input(G[0, 0], seed=7)[None]
    Gt, pt = torch.from_numpy(G).cuda(), torch.from_numpy(p).cuda()
    q_col = gf.fast_guided_filter(Gt.expand(1, 3, 300, 520).contiguous(), pt, 16, 3e-3, 4, "bilinear", color_guide=True)
    q_gray = gf.fast_guided_filter(Gt, pt, 16, 1e-3, 4, "bilinear")
    torch.cuda.synchronize()
    assert float((q_col - q_gray).abs().max()) <= 2 * TOL_F32


def test_self_guided_color_call_equals_copy(gf):
    I, _ = _inputs(1, 3, 128, 200, seed=8)
    It = torch.from_numpy(I).cuda()
    q_same = gf.fast_guided_filter(It, It, 8, 1e-2, 4, "bilinear", color_guide=True)
    q_copy = gf.fast_guided_filter(It, It.clone(), 8, 1e-2, 4, "bilinear", color_guide=True)
    torch.cuda.synchronize()
    assert torch.equal(q_same, q_copy)


def test_color_strips_equal_whole_image(gf):
    I, p = _inputs(1, 3, 700, 900, seed=9)
    It, pt = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    whole = gf.fast_guided_filter(It, pt, 16, 1e-3, 4, "bilinear", color_guide=True)
    q = torch.full_like(whole, float("nan"))
    for rows in gf.row_strips(700, 3):
        gf.fast_guided_filter(It, pt, 16, 1e-3, 4, "bilinear", color_guide=True, out=q, rows=rows)
    torch.cuda.synchronize()
    assert not torch.isnan(q).any()
    assert float((q - whole).abs().max()) <= 2 * TOL_F32


def test_color_feathering_12mp_sampled_rows(gf):
    """Fig. 4: a colour image guides a coarse binary mask, r = 60 (r' = 15), eps = 0.001^2, s = 4, 12 MP."""
    H, W, r, eps, s = 3000, 4000, 60, 0.001 ** 2, 4
    I = synth.make_color_scene(H, W, seed=10)[None]
    m = synth.feather_mask(H, W, seed=11)[None, None]
    got = _gpu(gf, I, m, r, eps, s, "bilinear")
    rl = oracle.lowres_radius(r, s)
    margin = s * (2 * rl + 4)
    for Y0 in (0, 1496, 2990):
        Y1 = min(H, Y0 + 10)
        ys, ye = max(0, Y0 - margin) // s * s, min(H, Y1 + margin)
        ref = oracle.color_guided_filter(I[..., ys:ye, :].astype(np.float64), m[..., ys:ye, :].astype(np.float64),
                                         r, eps, s, oracle.SUB_BILINEAR, r_low=rl)
        err = max_abs(got[..., Y0:Y1, :], ref[..., Y0 - ys:Y1 - ys, :])
        assert err <= TOL_F32, "rows %d..%d: max-abs error %.3g" % (Y0, Y1, err)


def test_color_guide_argument_checks(gf):
    o = gf.binding.opts_init()
    o.color_guide = 1
    o.guide_channels = 1
    n = ctypes.c_size_t()
    lib = gf.load_library()
    assert lib.gf_workspace_size(64, 64, 3, 4, ctypes.byref(o), ctypes.byref(n)) == gf.GF_EINVAL  # needs 3 channels
    o.guide_channels = 3
    assert lib.gf_workspace_size(64, 64, 3, 4, ctypes.byref(o), ctypes.byref(n)) == gf.GF_OK
    assert lib.gf_filter_kernel_count(64, 64, 3, 4, gf.GF_SUB_BILINEAR, ctypes.byref(o)) == 6
    o.dtype_in = gf.GF_U8
    assert lib.gf_workspace_size(64, 64, 3, 4, ctypes.byref(o), ctypes.byref(n)) == gf.GF_EINVAL
    I = torch.rand(1, 3, 32, 32, device="cuda")
    with pytest.raises(gf.GFError) as ei:  # forward only
        o2 = gf.binding.opts_init()
        o2.guide_channels, o2.color_guide = 3, 1
        ctx = gf.binding.default_context(0)
        g = torch.empty_like(I)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        gf.binding.check(lib.gf_filter_backward(ctx.handle, ptr(I), ptr(I), ptr(I), ptr(g), ptr(g), None, 32, 32, 3,
                                                4, 1e-2, 4, gf.GF_SUB_BILINEAR, ctypes.byref(o2), None))
    assert ei.value.status == gf.GF_EINVAL
