"""Row strips (gf_opts.row_begin / row_end) on the GPU: one image split into strips that are filtered
independently, here as "virtual devices" -- one CUDA stream per strip on one GPU, no data exchanged.

Checks: every row is written by its own strip and rows outside a strip are left untouched; the strips
agree with the whole-image call to within twice the parity tolerance (both are FP32 evaluations of the
same exact result, tiled from different first rows, so their rounding differs); and the strips match the
FP64 oracle within the parity tolerance, on every pixel at small sizes and on the rows around each strip
edge at 12 MP.  Covers every subsample mode, s = 1, 2, 4, 8, FP16
and uint8 storage, depthwise guides, a low-res p, the detail epilogue, and strip edges that do not fall on
multiples of s.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import TOL_F16, TOL_F32, max_abs, oracle_q, oracle_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _strips_on_streams(gf, I, p, q, strips, **kw):
    streams = [torch.cuda.Stream() for _ in strips]
    torch.cuda.synchronize()
    ctxs = [gf.Context() for _ in strips]  # own scratch per strip, as on separate devices
    for st, cx, rows in zip(streams, ctxs, strips):
        gf.fast_guided_filter(I, p, out=q, rows=rows, stream=st, ctx=cx, **kw)
    torch.cuda.synchronize()
    for cx in ctxs:
        cx.close()
    return q


CASES = [  # (H, W, C, CI, r, eps, s, mode, dtype, strips, extra)
    (3000, 4000, 3, 1, 16, 1e-3, 4, "bilinear", torch.float32, 2, {}),        # the 12 MP workload, 2 devices
    (3000, 4000, 3, 1, 16, 1e-3, 4, "bilinear", torch.float32, 8, {}),
    (1000, 1500, 3, 1, 16, 1e-3, 1, "bilinear", torch.float32, 3, {}),
    (1001, 1504, 1, 1, 64, 1e-3, 8, "nearest", torch.float32, 3, {}),
    (777, 640, 3, 3, 8, 1e-2, 2, "box", torch.float32, 4, {}),
    (600, 800, 3, 1, 12, 1e-2, 4, "bilinear", torch.float16, 3, {}),
    (600, 800, 3, 1, 12, 1e-2, 4, "bilinear", torch.uint8, 3, {}),
    (480, 640, 3, 3, 16, 1e-2, 4, "bilinear", torch.float32, 2, {"detail_gain": 5.0}),
    (512, 512, 3, 3, 0, 1e-2, 4, "box", torch.float32, 3, {"r_low": 2, "p_lowres": True}),
    (700, 900, 3, 1, 16, 1e-3, 4, "bilinear_aa", torch.float32, 3, {}),
    (701, 640, 1, 1, 24, 1e-3, 8, "bilinear_aa", torch.float16, 2, {}),
]


def _make(H, W, C, CI, s, dtype, extra, seed):
    I = synth.make_color_scene(H, W, seed=seed)[:CI] if CI > 1 else synth.make_scene(H, W, seed=seed)[None]
    if extra.get("p_lowres"):
        p = np.random.default_rng(seed + 1).uniform(0, 1, (C, -(-H // s), -(-W // s))).astype(np.float32)
    else:
        p = synth.rgb_noisy_input(I[0], seed=seed + 1, channels=C)
    It, pt = torch.from_numpy(I[None]).cuda(), torch.from_numpy(p[None]).cuda()
    if dtype == torch.uint8:
        It, pt = (It * 255).round().to(torch.uint8), (pt * 255).round().to(torch.uint8)
    else:
        It, pt = It.to(dtype), pt.to(dtype)
    return It, pt


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%dx%d_C%d_CI%d_r%d_s%d_%s_%s_x%d%s" % (
    c[0], c[1], c[2], c[3], c[4], c[6], c[7], str(c[8]).split(".")[-1], c[9], "_" + "_".join(c[10]) if c[10] else ""))
def test_strips_equal_whole_image(gf, case):
    H, W, C, CI, r, eps, s, mode, dtype, n, extra = case
    I, p = _make(H, W, C, CI, s, dtype, extra, seed=H + W)
    whole = gf.fast_guided_filter(I, p, r, eps, s, mode, **extra)
    q = torch.full_like(whole, float("nan"))
    strips = gf.row_strips(H, n, align=1 if n > 2 else 4 * s + 1)  # edges off the multiples of s
    _strips_on_streams(gf, I, p, q, strips, r=r, eps=eps, s=s, mode=mode, **extra)
    assert not torch.isnan(q).any()  # every row written by its strip
    tol = (TOL_F16 if dtype == torch.float16 else TOL_F32) * max(1.0, abs(1.0 - extra.get("detail_gain", 0.0)))
    assert float((q.float() - whole.float()).abs().max()) <= 2 * tol
    # the rows around every strip edge against the oracle (on the values actually stored)
    Ih = I.cpu().numpy().astype(np.float64) / (255.0 if dtype == torch.uint8 else 1.0)
    ph = p.cpu().numpy().astype(np.float64) / (255.0 if dtype == torch.uint8 else 1.0)
    modes = {"nearest": oracle.SUB_NEAREST, "bilinear": oracle.SUB_BILINEAR, "box": oracle.SUB_BOX,
             "bilinear_aa": oracle.SUB_BILINEAR_AA}
    if extra.get("p_lowres"):
        ref = oracle.fast_guided_filter(Ih, ph, r, eps, s, modes[mode], r_low=extra["r_low"], p_lowres=True)
    elif H * W <= 1_000_000:
        ref = oracle.fast_guided_filter(Ih, ph, r, eps, s, modes[mode])
    else:
        ref = None
    for _, edge in strips[:-1]:
        Y0, Y1 = max(0, edge - 3), min(H, edge + 3)
        want = ref[..., Y0:Y1, :] if ref is not None else oracle_rows(Ih, ph, Y0, Y1, r, eps, s, modes[mode])
        if extra.get("detail_gain"):
            want = oracle.detail_enhance(Ih[..., Y0:Y1, :], want, extra["detail_gain"])
        assert max_abs(q[..., Y0:Y1, :].float().cpu().numpy(), want) <= tol


def test_rows_outside_the_strip_are_untouched(gf):
    H, W = 400, 600
    I, p = _make(H, W, 3, 1, 4, torch.float32, {}, seed=3)
    for rows in ((0, 1), (123, 250), (399, 400), (0, 400)):
        q = torch.full((1, 3, H, W), float("nan"), device="cuda")
        gf.fast_guided_filter(I, p, 16, 1e-3, 4, "bilinear", out=q, rows=rows)
        torch.cuda.synchronize()
        inside = q[:, :, rows[0]:rows[1]]
        assert not torch.isnan(inside).any()
        assert int((~torch.isnan(q)).sum()) == inside.numel()


def test_strip_matches_oracle(gf):
    H, W, r, eps, s = 300, 520, 16, 1e-3, 4
    I, p = _make(H, W, 3, 1, s, torch.float32, {}, seed=5)
    q = torch.zeros((1, 3, H, W), device="cuda")
    gf.fast_guided_filter(I, p, r, eps, s, "bilinear", out=q, rows=(101, 207))
    torch.cuda.synchronize()
    ref = oracle_q(I.cpu().numpy(), p.cpu().numpy(), r, eps, s, oracle.SUB_BILINEAR)
    assert max_abs(q[..., 101:207, :].cpu().numpy(), ref[..., 101:207, :]) <= TOL_F32
