"""The single-kernel form (gf_opts.fused) on the GPU: Algorithm 2 in one kernel per output tile, each CTA
recomputing the halo of subsampled input, statistics and coefficients it needs.

Checks against the FP64 oracle: a 2 MP image (larger than the automatic threshold, forced), the plain
guided filter at s = 1 (the 512 x 512 workload), depthwise guides, FP16 storage, every subsample mode and a
non-integer ratio, the detail epilogue, and row strips; the automatic choice (one kernel below
GF_FUSED_AUTO_PIXELS, four above); and the argument checks of a forced fused call.  Tolerance TOL_F32
(TOL_F16 for FP16 storage).
"""
import ctypes
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import TOL_F16, TOL_F32, max_abs, oracle_q

pytestmark = pytest.mark.gpu

MODES = {"nearest": 0, "bilinear": 1, "box": 2, "bilinear_aa": 3}


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _scene(N, CI, C, H, W, seed):
    I = np.stack([synth.make_color_scene(H, W, seed=seed + k)[:CI] if CI > 1 else synth.make_scene(H, W, seed=seed + k)[None]
                  for k in range(N)])
    p = np.clip(I[:, :1] + np.random.default_rng(seed).normal(0, 0.1, (N, C, H, W)), 0, 1).astype(np.float32)
    return I.astype(np.float32), p


CASES = [  # (N, CI, C, H, W, r, eps, s, mode)
    (1, 1, 3, 1080, 1920, 8, 1e-3, 4, "bilinear"),    # 2 MP: above the automatic threshold, forced
    (1, 1, 1, 512, 512, 8, 1e-2, 1, "nearest"),       # the plain guided filter (Algorithm 1) in one kernel
    (2, 3, 3, 200, 264, 8, 1e-2, 4, "box"),           # depthwise guide, batch
    (1, 1, 2, 301, 411, 12, 1e-3, 3, "nearest"),      # odd s, ragged tiles
    (1, 1, 1, 256, 384, 16, 1e-3, 8, "bilinear_aa"),
    (1, 1, 3, 250, 330, 10, 1e-2, Fraction(5, 2), "bilinear"),
    (1, 1, 1, 37, 53, 60, 1e-6, 4, "bilinear"),       # r' = 15: windows wider than the image
    (1, 1, 1, 5, 3, 2, 1e-2, 2, "bilinear"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%dCI%dC%d_%dx%d_r%d_s%s_%s" % (
    c[0], c[1], c[2], c[3], c[4], c[5], str(c[7]).replace("/", "o"), c[8]))
def test_fused_parity(gf, case):
    N, CI, C, H, W, r, eps, s, mode = case
    I, p = _scene(N, CI, C, H, W, seed=H + W)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, mode, fused=1)
    torch.cuda.synchronize()
    ref = oracle_q(I, p, r, eps, s, MODES[mode])
    err = max_abs(q.cpu().numpy(), ref)
    assert err <= TOL_F32, "max-abs error %.3g" % err


def test_fused_fp16_and_detail(gf):
    I, _ = _scene(1, 3, 3, 240, 320, seed=5)
    I16 = I.astype(np.float16)
    q = gf.fast_guided_filter(torch.from_numpy(I16).cuda(), torch.from_numpy(I16).cuda(), 16, 0.1 ** 2, 4, "bilinear",
                              detail_gain=5.0, fused=1)
    torch.cuda.synchronize()
    q64 = oracle_q(I16.astype(np.float64), I16.astype(np.float64), 16, 0.1 ** 2, 4, 1)
    ref = oracle.detail_enhance(I16.astype(np.float64), q64, 5.0)
    assert max_abs(q.float().cpu().numpy(), ref) <= 4 * TOL_F16


def test_fused_strips_and_chain_agree(gf):
    I, p = _scene(1, 1, 3, 600, 800, seed=6)
    It, pt = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    chain = gf.fast_guided_filter(It, pt, 16, 1e-3, 4, "bilinear", fused=-1)
    q = torch.full_like(chain, float("nan"))
    for rows in gf.row_strips(600, 3):
        gf.fast_guided_filter(It, pt, 16, 1e-3, 4, "bilinear", out=q, rows=rows, fused=1)
    torch.cuda.synchronize()
    assert not torch.isnan(q).any()
    assert float((q - chain).abs().max()) <= 2 * TOL_F32


def test_automatic_choice_and_checks(gf):
    lib = gf.load_library()
    o = gf.binding.opts_init()
    count = lambda H, W, C: lib.gf_filter_kernel_count(H, W, C, 4, gf.GF_SUB_BILINEAR, ctypes.byref(o))
    assert count(512, 512, 3) == 1                    # small: one kernel
    assert count(1024, 1024, 1) == 1                  # N C H W = 2^20: still one
    assert count(1024, 1024, 3) == 4                  # above the threshold: the chain
    s1 = lib.gf_filter_kernel_count(256, 256, 1, 1, gf.GF_SUB_BILINEAR, ctypes.byref(o))
    assert s1 == 2                                    # s = 1: the chain (statistics, box means + output)
    o.fused = -1
    assert count(512, 512, 3) == 4
    o.fused = 1
    assert count(3000, 4000, 3) == 1
    o.dtype_in = gf.GF_U8                              # uint8 keeps its exact integer sums in the chain
    n = ctypes.c_size_t()
    assert lib.gf_workspace_size(64, 64, 1, 4, ctypes.byref(o), ctypes.byref(n)) == gf.GF_EINVAL
    o.dtype_in = gf.GF_F32
    o.r_low = 100                                      # too large a radius for the fused tiles
    assert lib.gf_workspace_size(64, 64, 1, 4, ctypes.byref(o), ctypes.byref(n)) == gf.GF_EINVAL
    I = torch.rand(1, 3, 64, 64, device="cuda")
    with pytest.raises(gf.GFError):
        gf.fast_guided_filter(I, I, 8, 1e-2, 4, "bilinear", color_guide=True, fused=1)
    # intermediate outputs are produced by the chain even when the image is small
    h, w, _ = gf.lowres_geometry(64, 64, 4, 8)
    a = torch.empty((1, 3, h, w), device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * gf.GF_MAX_STAGES)]
    gf.fast_guided_filter(I, I, 8, 1e-2, 4, "bilinear", a_out=a, kernel_events=ev)
    torch.cuda.synchronize()
    assert ev[6].elapsed_time(ev[7]) >= 0.0  # a fourth kernel ran
