"""GPU parity of the TMA-fed box kernels (csrc/gf_box.cu) against the FP64 oracle.

Those kernels take Algorithm 2's box statistics with the coefficients of Eq. 2-3, the box means of a and b,
and at s = 1 the box means fused with the output of Eq. 4 (the upsample is the identity there), when the
planes' rows are a multiple of 4 floats and r' <= 16 (16-row tiles up to r' = 8, 32-row tiles above).  Each
radius 0..16 is run at s = 1 and s = 4 on images whose tiles are all border tiles and on images with interior
tiles, with batch, depthwise guides, FP16 output, the detail epilogue and row ranges; the same calls with the
TMA kernels switched off (GF_NO_TMA_BOX: the per-thread-load kernels) must agree with the oracle too.
Tolerance: max-abs 1e-4 (FP32), 2e-3 (FP16).
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


@pytest.mark.parametrize("r", list(range(0, 17)))
def test_s1_every_radius(gf, r):
    """s = 1 (the plain guided filter, Algorithm 1): statistics and the fused box means + output, every
    compile-time radius and the run-time ones (0, 9..14); 70 x 132 has only border tiles."""
    I = _rand((1, 1, 70, 132), 10 + r)
    p = _rand((1, 2, 70, 132), 20 + r)
    q = _run(gf, I, p, r, 1e-2, 1)
    assert max_abs(q, oracle_q(I, p, r, 1e-2, 1, oracle.SUB_BILINEAR)) <= TOL_F32


@pytest.mark.parametrize("rl", list(range(0, 17)))
def test_s4_every_lowres_radius(gf, rl):
    """s = 4 with r' given explicitly: the statistics and box-mean kernels on a 70 x 132 low-res grid."""
    I = _rand((1, 1, 280, 528), 30 + rl)
    p = _rand((1, 3, 280, 528), 40 + rl)
    q = _run(gf, I, p, 4 * rl, 1e-3, 4, r_low=rl, fused=-1)
    ref = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), 4 * rl, 1e-3, 4,
                                    oracle.SUB_BILINEAR, r_low=rl)
    assert max_abs(q, ref) <= TOL_F32


@pytest.mark.parametrize("r,s", [(4, 1), (8, 1), (16, 1), (16, 4), (60, 4), (24, 8)])
def test_interior_tiles(gf, r, s):
    """Images with tiles away from every border (the unmasked path) next to border tiles."""
    H, W = (320, 400) if s == 1 else (160 * s, 200 * s)
    I = _rand((1, 1, H, W), 50 + r)
    p = _rand((1, 3, H, W), 60 + r)
    q = _run(gf, I, p, r, 1e-3, s, fused=-1)
    assert max_abs(q, oracle_q(I, p, r, 1e-3, s, oracle.SUB_BILINEAR)) <= TOL_F32


@pytest.mark.parametrize("case", [(2, 1, 3), (2, 3, 3), (3, 1, 1)], ids=["batch", "depthwise", "batch_gray"])
def test_batch_and_guides(gf, case):
    N, CI, C = case
    for s, r in ((1, 8), (4, 12)):
        I = _rand((N, CI, 96, 196), 70 + s)
        p = _rand((N, C, 96, 196), 80 + s)
        q = _run(gf, I, p, r, 1e-2, s, fused=-1)
        assert max_abs(q, oracle_q(I, p, r, 1e-2, s, oracle.SUB_BILINEAR)) <= TOL_F32


def test_s1_fp16_output_and_detail(gf):
    """The fused s = 1 output kernel stores FP16 q, and applies the detail epilogue q + k (I - q)."""
    I = _rand((1, 1, 64, 200), 90)
    p = _rand((1, 3, 64, 200), 91)
    q16 = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), 8, 1e-2, 1, "bilinear",
                                out_dtype=torch.float16)
    torch.cuda.synchronize()
    assert q16.dtype == torch.float16
    ref = oracle_q(I, p, 8, 1e-2, 1, oracle.SUB_BILINEAR)
    assert max_abs(q16.float().cpu().numpy(), ref) <= TOL_F16
    Ig = np.repeat(I, 3, axis=1)
    qd = _run(gf, Ig, Ig, 8, 1e-2, 1, detail_gain=5.0)
    base = oracle_q(Ig, Ig, 8, 1e-2, 1, oracle.SUB_BILINEAR)
    assert max_abs(qd, base + 5.0 * (Ig - base)) <= 6 * TOL_F32


def test_s1_row_range(gf):
    """A row range at s = 1 writes only its rows, equal to the whole-image call's."""
    I = _rand((1, 1, 150, 164), 92)
    p = _rand((1, 2, 150, 164), 93)
    full = _run(gf, I, p, 6, 1e-2, 1)
    Id, pd = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    q = torch.full_like(pd, -7.0)
    gf.fast_guided_filter(Id, pd, 6, 1e-2, 1, "bilinear", out=q, rows=(37, 101))
    torch.cuda.synchronize()
    q = q.cpu().numpy()
    assert np.all(q[..., :37, :] == -7.0) and np.all(q[..., 101:, :] == -7.0)
    assert max_abs(q[..., 37:101, :], full[..., 37:101, :]) <= 1e-5


def test_s1_kernel_count(gf):
    """s = 1 with rows of a multiple of 4 floats runs two kernels (statistics; box means + output): the
    call records two pairs of kernel events, and the third pair is left as it was."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * gf.GF_MAX_STAGES)]
    marker = torch.cuda.Event(enable_timing=True)
    I = _rand((1, 1, 64, 128), 94)
    x = torch.zeros(1, device="cuda")
    for e in ev[4:6]:
        e.record()  # recorded before the call
    x += 1
    marker.record()
    _run(gf, I, I, 8, 1e-2, 1, kernel_events=ev)
    for k in range(2):
        assert ev[2 * k].elapsed_time(ev[2 * k + 1]) >= 0.0
        assert marker.elapsed_time(ev[2 * k]) >= 0.0   # recorded by the call
    assert ev[4].elapsed_time(marker) >= 0.0            # still the record from before the call


@pytest.mark.parametrize("s,r,W", [(1, 16, 300), (4, 16, 704), (1, 8, 301), (4, 24, 702)])
def test_with_and_without_tma(gf, monkeypatch, s, r, W):
    """The same call through the TMA kernels and through the per-thread-load kernels (GF_NO_TMA_BOX, read per
    call): both within the tolerance of the oracle (W % 4 != 0 takes the second form either way)."""
    I = _rand((1, 1, 120, W), 95)
    p = _rand((1, 3, 120, W), 96)
    ref = oracle_q(I, p, r, 1e-3, s, oracle.SUB_BILINEAR)
    q1 = _run(gf, I, p, r, 1e-3, s, fused=-1)
    monkeypatch.setenv("GF_NO_TMA_BOX", "1")
    q2 = _run(gf, I, p, r, 1e-3, s, fused=-1)
    monkeypatch.delenv("GF_NO_TMA_BOX")
    assert max_abs(q1, ref) <= TOL_F32 and max_abs(q2, ref) <= TOL_F32


def test_intermediates_through_tma(gf):
    """a, b, their box means and the window means written by the TMA kernels into caller buffers (w % 4 == 0)
    match the oracle's intermediates."""
    H, W, r, eps, s = 128, 512, 16, 1e-2, 4
    I = _rand((1, 1, H, W), 97)
    p = _rand((1, 2, H, W), 98)
    h, w, rl = gf.lowres_geometry(H, W, s, r)
    dev = torch.device("cuda")
    a = torch.empty((1, 2, h, w), device=dev)
    b, ma, mb = torch.empty_like(a), torch.empty_like(a), torch.empty_like(a)
    st = torch.empty((1, 2, 4, h, w), device=dev)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, "bilinear",
                              a_out=a, b_out=b, mean_a_out=ma, mean_b_out=mb, stats_out=st, fused=-1)
    torch.cuda.synchronize()
    ref_q, inter = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), r, eps, s,
                                             oracle.SUB_BILINEAR, intermediates=True)
    assert max_abs(q.cpu(), ref_q) <= TOL_F32
    assert max_abs(st.cpu(), inter["stats"]) <= 2e-6  # mean_I, corr_I, mean_p, corr_Ip
    # an absolute error e in the window statistics moves a by about e / eps
    tol = 2e-6 / eps * 10
    assert max_abs(a.cpu(), inter["a"]) <= tol and max_abs(b.cpu(), inter["b"]) <= tol
    assert max_abs(ma.cpu(), inter["mean_a"]) <= tol and max_abs(mb.cpu(), inter["mean_b"]) <= tol


@pytest.mark.parametrize("fused", [-1, 1], ids=["chain", "single_kernel"])
@pytest.mark.parametrize("W", [528, 530], ids=["tma", "per_thread_loads"])
@pytest.mark.parametrize("mode", ["nearest", "bilinear"])
def test_one_sample_window_is_exact(gf, mode, W, fused):
    """r' = 0 (one-sample windows): var_I = cov_Ip = 0 exactly, so Eq. 2 gives a = 0 and q is the upsampled
    box mean of p' whatever eps; with a tiny eps any rounding left in var or cov would be amplified by 1 / eps.
    Every statistics kernel (TMA tiles, per-thread loads, the single fused kernel)."""
    m = {"nearest": oracle.SUB_NEAREST, "bilinear": oracle.SUB_BILINEAR}[mode]
    I = _rand((1, 1, 280, W), 500)
    p = _rand((1, 3, 280, W), 501)
    q = _run(gf, I, p, 0, 1e-6, 4, mode, r_low=0, fused=fused)
    ref = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), 0, 1e-6, 4, m, r_low=0)
    assert max_abs(q, ref) <= TOL_F32
