"""GPU parity of the fused subsample + box statistics kernel (k_box_strip_sub, csrc/gf_strip.cu) against the
FP64 oracle.

That kernel takes Algorithm 2's first two steps in one pass for a gray guide serving three channels at
r' = 4, s = 4 or 8, nearest or bilinear: TMA streams the full-res rows each low-res sample reads into shared
memory, each walker forms its column's samples there (the subsample's arithmetic) and sums them into the
window, and the column-strip statistics' phase 2 applies Eq. 2-3.  It is an opt-in form (GF_SUB_STRIP=1),
so every case here sets that variable and checks that the call really ran three kernels.  The cases span
several 128-column strips with a ragged last one, several row segments, planes narrower than a strip and
shorter than a block of 10 rows, a batch, two channel groups, the intermediates a and b in caller buffers,
and the chain's own result on the same inputs.  Tolerance: max-abs 1e-4 (FP32).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import TOL_F32, max_abs, oracle_q

pytestmark = pytest.mark.gpu

MODES = {"bilinear": oracle.SUB_BILINEAR, "nearest": oracle.SUB_NEAREST}


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


@pytest.fixture
def fused_sub(monkeypatch):
    monkeypatch.setenv("GF_SUB_STRIP", "1")


def _rand(shape, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, shape).astype(np.float32)


def _run(gf, I, p, r, eps, s, mode, **kw):
    """The filter through the library, with the kernel count of the call checked: three stages ran (the
    fused kernel, the box means, the output) and the fourth stage's events were never recorded."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * gf.GF_MAX_STAGES)]
    x = torch.zeros(1, device="cuda")
    for e in ev[6:8]:
        e.record()
    x += 1
    marker = torch.cuda.Event(enable_timing=True)
    marker.record()
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, mode,
                              kernel_events=ev, fused=-1, **kw)
    torch.cuda.synchronize()
    for k in range(3):
        assert marker.elapsed_time(ev[2 * k]) >= 0.0
    assert ev[6].elapsed_time(marker) >= 0.0  # no fourth kernel
    return q.float().cpu().numpy()


@pytest.mark.parametrize("mode", ["bilinear", "nearest"])
@pytest.mark.parametrize("s", [4, 8])
def test_strips_and_segments(gf, fused_sub, s, mode):
    """3 strips (the last 16 low-res columns wide), several segments, a ragged last block of rows."""
    H, W = 10 * 23 * s // 2, 272 * s  # h = 115, w = 272
    H -= H % s
    I = _rand((1, 1, H, W), 600 + s)
    p = _rand((1, 3, H, W), 610 + s)
    q = _run(gf, I, p, 4 * s, 1e-3, s, mode)
    assert max_abs(q, oracle_q(I, p, 4 * s, 1e-3, s, MODES[mode])) <= TOL_F32


@pytest.mark.parametrize("H,W", [(32, 64), (8, 16), (44, 512), (4096, 128)])
def test_small_and_tall_planes(gf, fused_sub, H, W):
    """Planes narrower than a strip, shorter than a block, exactly one strip wide, and tall (many segments)."""
    I = _rand((1, 1, H, W), 620 + H)
    p = _rand((1, 3, H, W), 630 + W)
    q = _run(gf, I, p, 16, 1e-2, 4, "bilinear")
    assert max_abs(q, oracle_q(I, p, 16, 1e-2, 4, oracle.SUB_BILINEAR)) <= TOL_F32


def test_batch_and_two_groups(gf, fused_sub):
    """N = 2 images of C = 6 channels under one gray guide each: two groups of three channels per image."""
    I = _rand((2, 1, 160, 1056), 640)
    p = _rand((2, 6, 160, 1056), 641)
    q = _run(gf, I, p, 16, 1e-3, 4, "bilinear")
    assert max_abs(q, oracle_q(I, p, 16, 1e-3, 4, oracle.SUB_BILINEAR)) <= TOL_F32


def test_intermediates(gf, fused_sub):
    """a and b, written by the fused kernel into caller buffers, and their box means match the oracle's."""
    H, W, r, eps, s = 240, 1040, 16, 1e-2, 4
    I = _rand((1, 1, H, W), 650)
    p = _rand((1, 3, H, W), 651)
    h, w, rl = gf.lowres_geometry(H, W, s, r)
    assert rl == 4
    dev = torch.device("cuda")
    a = torch.empty((1, 3, h, w), device=dev)
    b, ma, mb = torch.empty_like(a), torch.empty_like(a), torch.empty_like(a)
    q = _run(gf, I, p, r, eps, s, "bilinear", a_out=a, b_out=b, mean_a_out=ma, mean_b_out=mb)
    ref_q, inter = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), r, eps, s,
                                             oracle.SUB_BILINEAR, intermediates=True)
    assert max_abs(q, ref_q) <= TOL_F32
    tol = 2e-6 / eps * 10  # an absolute error e in the window statistics moves a by about e / eps
    assert max_abs(a.cpu(), inter["a"]) <= tol and max_abs(b.cpu(), inter["b"]) <= tol
    assert max_abs(ma.cpu(), inter["mean_a"]) <= tol and max_abs(mb.cpu(), inter["mean_b"]) <= tol


def test_agrees_with_the_chain(gf, monkeypatch):
    """The same call with and without the fused kernel: both within rounding of each other (the window sums
    are taken over different row segments, so they are not bit-identical)."""
    I = _rand((1, 1, 600, 2048), 660)
    p = _rand((1, 3, 600, 2048), 661)
    monkeypatch.setenv("GF_SUB_STRIP", "1")
    q1 = _run(gf, I, p, 16, 1e-3, 4, "bilinear")
    monkeypatch.delenv("GF_SUB_STRIP")
    q0 = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), 16, 1e-3, 4, "bilinear",
                               fused=-1).float().cpu().numpy()
    assert max_abs(q1, q0) <= TOL_F32
