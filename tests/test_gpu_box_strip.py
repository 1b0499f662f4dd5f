"""GPU parity of the column-strip box kernels (csrc/gf_strip.cu) against the FP64 oracle.

Those kernels take the box steps at radii 9..16 (Algorithm 1 at s = 1, Algorithm 2's low-res box steps at
s > 1): the statistics with the coefficients of Eq. 2-3 -- one CTA for the three channels of a gray guide,
else one per channel --, the box means of a and b, and at s = 1 the box means fused with Eq. 4.  A CTA owns a
strip of 128 output columns over a segment of at most 160 rows, so the cases below span several strips with a
ragged last one, several segments, images narrower than a strip and shorter than a block of 10 rows, batches,
two channel groups, depthwise guides, FP16 output, the detail epilogue, row ranges and the colour guide's box
steps; the same calls with the strip kernels switched off (GF_NO_STRIP_BOX: the tile kernels) must agree with
the oracle too.  Tolerance: max-abs 1e-4 (FP32), 2e-3 (FP16).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import TOL_F16, TOL_F32, max_abs, oracle_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _rand(shape, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, shape).astype(np.float32)


def _run(gf, I, p, r, eps, s, mode="bilinear", **kw):
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, mode, **kw)
    torch.cuda.synchronize()
    return q.float().cpu().numpy()


@pytest.mark.parametrize("r", list(range(9, 17)))
@pytest.mark.parametrize("CI,C", [(1, 3), (1, 2), (3, 3)], ids=["gray3", "gray2", "depthwise"])
def test_s1_radii(gf, r, CI, C):
    """s = 1, every strip radius: 3 strips (the last 44 columns wide), 2 segments, a ragged last block."""
    I = _rand((1, CI, 173, 300), 100 + r)
    p = _rand((1, C, 173, 300), 200 + r)
    q = _run(gf, I, p, r, 1e-3, 1)
    assert max_abs(q, oracle_q(I, p, r, 1e-3, 1, oracle.SUB_BILINEAR)) <= TOL_F32


@pytest.mark.parametrize("rl", [9, 12, 15, 16])
def test_lowres_radii(gf, rl):
    """s = 4 with r' = 9..16: the strip statistics and box-mean kernels on a 150 x 260 low-res grid."""
    I = _rand((1, 1, 600, 1040), 300 + rl)
    p = _rand((1, 3, 600, 1040), 310 + rl)
    q = _run(gf, I, p, 4 * rl, 1e-3, 4, r_low=rl, fused=-1)
    ref = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), 4 * rl, 1e-3, 4,
                                    oracle.SUB_BILINEAR, r_low=rl)
    assert max_abs(q, ref) <= TOL_F32


@pytest.mark.parametrize("H,W", [(7, 64), (3, 4), (10, 128), (31, 132), (11, 260)])
def test_small_planes(gf, H, W):
    """Planes narrower than a strip and shorter than a block or a window: every window clipped."""
    for r, CI, C in ((16, 1, 3), (9, 1, 1), (13, 2, 2)):
        I = _rand((1, CI, H, W), H * W + r)
        p = _rand((1, C, H, W), H * W + r + 1)
        q = _run(gf, I, p, r, 1e-2, 1)
        assert max_abs(q, oracle_q(I, p, r, 1e-2, 1, oracle.SUB_BILINEAR)) <= TOL_F32


def test_tall_many_segments(gf):
    """700 rows at r = 16: a small grid, so many short segments, each opening its own window and shift."""
    I = _rand((1, 1, 700, 256), 400)
    p = _rand((1, 3, 700, 256), 401)
    q = _run(gf, I, p, 16, 1e-3, 1)
    assert max_abs(q, oracle_q(I, p, 16, 1e-3, 1, oracle.SUB_BILINEAR)) <= TOL_F32


@pytest.mark.parametrize("case", [(2, 1, 3), (2, 1, 6), (2, 3, 3), (3, 1, 1)],
                         ids=["batch_gray3", "two_groups", "batch_depthwise", "batch_gray1"])
def test_batch_and_groups(gf, case):
    N, CI, C = case
    I = _rand((N, CI, 96, 388), 410 + C)
    p = _rand((N, C, 96, 388), 420 + C)
    for s, r in ((1, 12), (4, 40)):
        q = _run(gf, I, p, r, 1e-2, s, fused=-1)
        assert max_abs(q, oracle_q(I, p, r, 1e-2, s, oracle.SUB_BILINEAR)) <= TOL_F32


def test_s1_fp16_output_and_detail(gf):
    """The strip box means + output kernel stores FP16 q and applies the detail epilogue q + k (I - q)."""
    I = _rand((1, 1, 64, 200), 430)
    p = _rand((1, 3, 64, 200), 431)
    q16 = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), 16, 1e-2, 1, "bilinear",
                                out_dtype=torch.float16)
    torch.cuda.synchronize()
    assert q16.dtype == torch.float16
    assert max_abs(q16.float().cpu().numpy(), oracle_q(I, p, 16, 1e-2, 1, oracle.SUB_BILINEAR)) <= TOL_F16
    Ig = np.repeat(I, 3, axis=1)
    qd = _run(gf, Ig, Ig, 11, 1e-2, 1, detail_gain=5.0)
    base = oracle_q(Ig, Ig, 11, 1e-2, 1, oracle.SUB_BILINEAR)
    assert max_abs(qd, base + 5.0 * (Ig - base)) <= 6 * TOL_F32


def test_s1_row_range(gf):
    """A row range at s = 1 (the strip kernel's segments start at the range's first row) writes only its
    rows, equal to the whole-image call's."""
    I = _rand((1, 1, 350, 164), 440)
    p = _rand((1, 2, 350, 164), 441)
    full = _run(gf, I, p, 14, 1e-2, 1)
    Id, pd = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    q = torch.full_like(pd, -7.0)
    gf.fast_guided_filter(Id, pd, 14, 1e-2, 1, "bilinear", out=q, rows=(37, 301))
    torch.cuda.synchronize()
    q = q.cpu().numpy()
    assert np.all(q[..., :37, :] == -7.0) and np.all(q[..., 301:, :] == -7.0)
    assert max_abs(q[..., 37:301, :], full[..., 37:301, :]) <= 1e-5


@pytest.mark.parametrize("s,r", [(1, 16), (1, 10), (4, 60), (2, 26)])
def test_with_and_without_strip(gf, monkeypatch, s, r):
    """The same call through the strip kernels and through the tile kernels (GF_NO_STRIP_BOX, read per call):
    both within the tolerance of the oracle, and within 2e-5 of each other."""
    I = _rand((1, 1, 240, 520), 450 + r)
    p = _rand((1, 3, 240, 520), 460 + r)
    ref = oracle_q(I, p, r, 1e-3, s, oracle.SUB_BILINEAR)
    q1 = _run(gf, I, p, r, 1e-3, s, fused=-1)
    monkeypatch.setenv("GF_NO_STRIP_BOX", "1")
    q2 = _run(gf, I, p, r, 1e-3, s, fused=-1)
    monkeypatch.delenv("GF_NO_STRIP_BOX")
    assert max_abs(q1, ref) <= TOL_F32 and max_abs(q2, ref) <= TOL_F32
    assert max_abs(q1, q2) <= 2e-5


def test_intermediates_large_radius(gf):
    """a, b and their box means written by the strip kernels (s = 4, r' = 12) into caller buffers match the
    oracle's intermediates."""
    H, W, r, eps, s = 240, 1040, 48, 1e-2, 4
    I = _rand((1, 1, H, W), 470)
    p = _rand((1, 3, H, W), 471)
    h, w, rl = gf.lowres_geometry(H, W, s, r)
    assert rl == 12
    dev = torch.device("cuda")
    a = torch.empty((1, 3, h, w), device=dev)
    b, ma, mb = torch.empty_like(a), torch.empty_like(a), torch.empty_like(a)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, "bilinear",
                              a_out=a, b_out=b, mean_a_out=ma, mean_b_out=mb, fused=-1)
    torch.cuda.synchronize()
    ref_q, inter = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), r, eps, s,
                                             oracle.SUB_BILINEAR, intermediates=True)
    assert max_abs(q.cpu(), ref_q) <= TOL_F32
    tol = 2e-6 / eps * 10  # an absolute error e in the window statistics moves a by about e / eps
    assert max_abs(a.cpu(), inter["a"]) <= tol and max_abs(b.cpu(), inter["b"]) <= tol
    assert max_abs(ma.cpu(), inter["mean_a"]) <= tol and max_abs(mb.cpu(), inter["mean_b"]) <= tol


def test_s1_kernel_count(gf):
    """s = 1 at r = 16 still runs two kernels (strip statistics; strip box means + output)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * gf.GF_MAX_STAGES)]
    marker = torch.cuda.Event(enable_timing=True)
    I = _rand((1, 1, 64, 256), 480)
    x = torch.zeros(1, device="cuda")
    for e in ev[4:6]:
        e.record()
    x += 1
    marker.record()
    _run(gf, I, np.repeat(I, 3, axis=1), 16, 1e-2, 1, kernel_events=ev)
    for k in range(2):
        assert ev[2 * k].elapsed_time(ev[2 * k + 1]) >= 0.0
        assert marker.elapsed_time(ev[2 * k]) >= 0.0
    assert ev[4].elapsed_time(marker) >= 0.0


@pytest.mark.parametrize("s,r", [(1, 12), (4, 64)])
def test_color_guide_box_steps(gf, s, r):
    """The colour-guided form's box means (products, then coefficients) through the strip kernel (r' = 12, 16)."""
    import synth
    I = synth.make_color_scene(200, 520, seed=490)[None]
    p = np.clip(I + np.random.default_rng(491).normal(0, 0.1, I.shape), 0, 1).astype(np.float32)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, 1e-3, s, "bilinear",
                              color_guide=True)
    torch.cuda.synchronize()
    ref = oracle.color_guided_filter(I.astype(np.float64), p.astype(np.float64), r, 1e-3, s, oracle.SUB_BILINEAR)
    assert max_abs(q.cpu().numpy(), ref) <= TOL_F32


@pytest.mark.parametrize("r", list(range(1, 9)))
def test_small_radii_through_strips(gf, monkeypatch, r):
    """Radii 1..8 through the strip kernels (GF_STRIP_MIN_R=1, read per call) at s = 1 and s = 4: the windows
    narrower than a block of 8 columns and the run-time radius path."""
    monkeypatch.setenv("GF_STRIP_MIN_R", "1")
    I = _rand((1, 1, 173, 300), 600 + r)
    p = _rand((1, 3, 173, 300), 610 + r)
    q = _run(gf, I, p, r, 1e-3, 1)
    assert max_abs(q, oracle_q(I, p, r, 1e-3, 1, oracle.SUB_BILINEAR)) <= TOL_F32
    I4 = _rand((1, 2, 280, 520), 620 + r)
    p4 = _rand((1, 2, 280, 520), 630 + r)
    q4 = _run(gf, I4, p4, 4 * r, 1e-3, 4, r_low=r, fused=-1)
    ref4 = oracle.fast_guided_filter(I4.astype(np.float64), p4.astype(np.float64), 4 * r, 1e-3, 4,
                                     oracle.SUB_BILINEAR, r_low=r)
    assert max_abs(q4, ref4) <= TOL_F32
