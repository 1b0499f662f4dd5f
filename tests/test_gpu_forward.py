"""GPU parity of the forward path (libgf.so through the C ABI) against the FP64 oracle.

Every case runs the CUDA kernels through ``gf_filter`` and compares element by element with the oracle on
the same seeded inputs: tiny, ragged and multi-tile shapes, every subsample mode and ratio, batch and
depthwise guides, the 512 x 512 and 12 MP workloads, and the intermediates (a, b, their means, the window
statistics).  Tolerance: max-abs 1e-4 on [0, 1] data for FP32 (2e-3 for FP16 storage).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import TOL_F16, TOL_F32, max_abs, oracle_q, oracle_rows

pytestmark = pytest.mark.gpu

MODE_NAMES = {0: "nearest", 1: "bilinear", 2: "box", 3: "bilinear_aa"}


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _rand(shape, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, shape).astype(np.float32)


def _run(gf, I, p, r, eps, s, mode, **kw):
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, MODE_NAMES[mode], **kw)
    torch.cuda.synchronize()
    return q.float().cpu().numpy()


CASES = [
    # (N, CI, C, H, W, r, eps, s, mode)
    (1, 1, 1, 1, 1, 1, 1e-2, 1, 1),
    (1, 1, 1, 1, 37, 3, 1e-2, 1, 1),
    (1, 1, 1, 29, 1, 3, 1e-2, 2, 0),
    (1, 1, 2, 5, 7, 8, 1e-2, 1, 1),         # r' larger than the image
    (1, 1, 1, 9, 13, 0, 1e-2, 1, 1),        # r' = 0
    (1, 1, 3, 37, 53, 4, 1e-2, 2, 1),
    (1, 1, 1, 61, 43, 6, 1e-3, 3, 0),       # odd s, ragged
    (1, 1, 1, 61, 43, 6, 1e-3, 3, 1),
    (1, 1, 2, 66, 70, 8, 1e-3, 4, 2),       # box mode, ragged
    (1, 1, 3, 300, 701, 8, 1e-3, 2, 1),     # scalar path (W % 4 != 0), several strips and chunks
    (1, 1, 3, 300, 704, 16, 1e-3, 4, 1),    # vector path
    (1, 1, 3, 257, 1030, 16, 1e-3, 8, 0),
    (2, 1, 3, 96, 128, 8, 1e-2, 4, 1),      # batch
    (2, 3, 3, 96, 128, 8, 1e-2, 4, 2),      # depthwise guide
    (1, 1, 1, 200, 300, 16, 1e-3, 1, 1),    # plain guided filter, r = 16
    (1, 1, 1, 150, 420, 120, 1e-3, 1, 1),   # r = 120: large radius, compensated sums
    (1, 1, 2, 40, 1024, 60, 1e-6, 4, 1),    # paper's feathering radius (r' = 15), tiny eps
    (1, 1, 2, 203, 408, 16, 1e-3, 8, 1),    # s = 8 fast output path with a ragged last band
    (1, 1, 3, 120, 200, 8, 1e-3, 8, 1),     # s = 8 vector subsample + fast output, W % 8 == 0
    (1, 1, 3, 124, 204, 8, 1e-3, 8, 0),     # s = 8, W % 8 == 4: last 4-pixel group is a half cell
    (1, 1, 1, 64, 36, 4, 1e-2, 4, 0),       # narrower than one 512-pixel band
    (1, 1, 3, 128, 260, 6, 1e-2, 2, 1),     # s = 2 vector subsample
    (1, 1, 3, 130, 262, 6, 1e-2, 2, 0),     # s = 2, W % 4 != 0: generic paths
    (1, 1, 3, 97, 1300, 9, 1e-3, 4, 1),     # s = 4 fast output, H % 4 != 0, several bands across
    (1, 1, 1, 2000, 48, 40, 1e-3, 1, 1),    # s = 1, r = 40: compensated box sums
    # s = 4, 8 fast output path at its edges
    (1, 1, 3, 33, 68, 32, 1e-3, 4, 1),      # r' = 8, window wider than the image
    (1, 1, 1, 3, 4, 0, 1e-2, 4, 1),         # r' = 0, H < s, a single 4-pixel column
    (2, 1, 2, 130, 1028, 64, 1e-3, 8, 2),   # s = 8, r' = 8, box subsample, batch, ragged last band
    (1, 1, 3, 1000, 2052, 20, 1e-2, 4, 0),  # r' = 5, five bands, ragged
    # antialiased bilinear subsample (triangle filter of half-width s)
    (1, 1, 3, 300, 704, 16, 1e-3, 4, 3),
    (1, 1, 1, 61, 43, 6, 1e-3, 3, 3),       # odd s, ragged
    (2, 3, 3, 96, 128, 8, 1e-2, 4, 3),      # batch, depthwise guide
    (1, 1, 2, 203, 408, 16, 1e-3, 8, 3),    # s = 8, ragged last band
    (1, 1, 1, 7, 5, 4, 1e-2, 2, 3),         # tiny: every tap window clipped
    # vectorised FP32 box / antialiased subsample (H, W multiples of s)
    (1, 1, 2, 128, 256, 8, 1e-2, 2, 2),
    (2, 1, 3, 160, 320, 16, 1e-3, 8, 2),
    (1, 1, 1, 64, 64, 4, 1e-2, 2, 3),
    (1, 1, 2, 256, 512, 32, 1e-3, 8, 3),
    (1, 3, 3, 8, 8, 4, 1e-2, 4, 3),         # one low-res column and two rows: both borders in each
]


@pytest.mark.parametrize("fused", [-1, 0], ids=["chain", "auto"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%dCI%dC%d_%dx%d_r%d_s%d_m%d" % (c[0], c[1], c[2], c[3], c[4], c[5], c[7], c[8]))
def test_fp32_parity(gf, case, fused):
    """Every case through the four-kernel chain, and with the automatic choice (the single fused kernel for
    images up to GF_FUSED_AUTO_PIXELS where it takes the arguments)."""
    N, CI, C, H, W, r, eps, s, mode = case
    I = _rand((N, CI, H, W), 1 + H + W)
    p = _rand((N, C, H, W), 2 + H * W)
    q = _run(gf, I, p, r, eps, s, mode, fused=fused)
    ref = oracle_q(I, p, r, eps, s, mode)
    assert q.shape == ref.shape
    err = max_abs(q, ref)
    assert err <= TOL_F32, "max-abs error %.3g" % err


def test_intermediates_match_oracle(gf):
    N, C, H, W, r, eps, s, mode = 1, 3, 120, 260, 8, 1e-2, 4, 1
    I = synth.make_scene(H, W, seed=5)[None, None]
    p = synth.rgb_noisy_input(I[0, 0], seed=6)[None]
    h, w, rl = gf.lowres_geometry(H, W, s, r)
    dev = torch.device("cuda")
    a = torch.empty((N, C, h, w), device=dev)
    b = torch.empty_like(a)
    ma = torch.empty_like(a)
    mb = torch.empty_like(a)
    st = torch.empty((N, C, 4, h, w), device=dev)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, "bilinear",
                              a_out=a, b_out=b, mean_a_out=ma, mean_b_out=mb, stats_out=st)
    torch.cuda.synchronize()
    ref_q, inter = oracle.fast_guided_filter(I.astype(np.float64), p.astype(np.float64), r, eps, s, mode,
                                             intermediates=True)
    assert max_abs(q.cpu(), ref_q) <= TOL_F32
    assert max_abs(st.cpu(), inter["stats"]) <= 2e-6
    # a = cov / (var + eps): an absolute error e in var/cov moves a by about e / eps
    assert max_abs(a.cpu(), inter["a"]) <= 2e-6 / eps * 10
    assert max_abs(b.cpu(), inter["b"]) <= 2e-6 / eps * 10
    assert max_abs(ma.cpu(), inter["mean_a"]) <= 2e-6 / eps * 10
    assert max_abs(mb.cpu(), inter["mean_b"]) <= 2e-6 / eps * 10


def test_config0_512(gf):
    """512 x 512 scene (seed 0), p = I, r = 8, eps = 0.01, s = 4 nearest, and s = 1 on the same inputs."""
    I = synth.make_scene(512, 512, seed=0)
    for s, mode in ((4, 0), (1, 0)):
        q = _run(gf, I, I, 8, 0.01, s, mode)
        err = max_abs(q, oracle_q(I, I, 8, 0.01, s, mode))
        assert err <= TOL_F32, "s=%d err %.3g" % (s, err)


@pytest.fixture(scope="module")
def scene12mp():
    I = synth.make_scene(3000, 4000, seed=0)
    p = synth.rgb_noisy_input(I, seed=1)
    return I[None, None], p[None]


@pytest.mark.parametrize("s", [4, 8])
def test_config1_12mp_full_oracle(gf, scene12mp, s):
    """12 MP (4000 x 3000) gray guide, 3-channel noisy p, r = 16, eps = 1e-3, bilinear: every output."""
    I, p = scene12mp
    q = _run(gf, I, p, 16, 1e-3, s, 1)
    err = max_abs(q, oracle_q(I, p, 16, 1e-3, s, 1))
    assert err <= TOL_F32, "err %.3g" % err


def test_config1_12mp_s1_row_bands(gf, scene12mp):
    """12 MP at s = 1 (plain guided filter, r = 16): bands of rows at the top, middle and bottom, each
    compared exactly with the oracle run on a crop with enough margin."""
    I, p = scene12mp
    q = _run(gf, I, p, 16, 1e-3, 1, 1)
    H = I.shape[-2]
    for Y0, Y1 in ((0, 40), (1480, 1530), (H - 40, H)):
        ref = oracle_rows(I, p, Y0, Y1, 16, 1e-3, 1, 1)
        err = max_abs(q[..., Y0:Y1, :], ref)
        assert err <= TOL_F32, "rows %d-%d err %.3g" % (Y0, Y1, err)


def test_config1_12mp_antialiased_row_bands(gf, scene12mp):
    """12 MP, s = 4, antialiased bilinear subsample: bands of rows at the top, middle and bottom against
    the oracle on cropped rows (the crop margin covers the wider subsample taps)."""
    I, p = scene12mp
    q = _run(gf, I, p, 16, 1e-3, 4, 3)
    H = I.shape[-2]
    for Y0, Y1 in ((0, 40), (1480, 1530), (H - 40, H)):
        ref = oracle_rows(I, p, Y0, Y1, 16, 1e-3, 4, 3)
        err = max_abs(q[..., Y0:Y1, :], ref)
        assert err <= TOL_F32, "rows %d-%d err %.3g" % (Y0, Y1, err)


def test_output_guard_band(gf):
    """No write lands outside q: q is a view into a larger buffer whose margins hold a sentinel."""
    N, C, H, W = 1, 3, 50, 61
    I = _rand((N, 1, H, W), 3)
    p = _rand((N, C, H, W), 4)
    n = N * C * H * W
    big = torch.full((n + 2048,), 12345.0, device="cuda")
    out = big[1024:1024 + n].view(N, C, H, W)
    gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), 4, 1e-2, 2, "bilinear", out=out)
    torch.cuda.synchronize()
    assert torch.all(big[:1024] == 12345.0) and torch.all(big[1024 + n:] == 12345.0)
    assert max_abs(out.cpu(), oracle_q(I, p, 4, 1e-2, 2, 1)) <= TOL_F32


def test_fp16_storage(gf):
    I = synth.to_f16_values(synth.make_scene(600, 800, seed=7))
    p = synth.to_f16_values(synth.rgb_noisy_input(I.astype(np.float32), seed=8))
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), 16, 1e-3, 4, "bilinear")
    torch.cuda.synchronize()
    assert q.dtype == torch.float16
    ref = oracle_q(I.astype(np.float64), p.astype(np.float64), 16, 1e-3, 4, 1)
    assert max_abs(q.float().cpu(), ref) <= TOL_F16


@pytest.mark.parametrize("s,mode", [(4, 1), (4, 0), (1, 1), (3, 1), (8, 1)])
def test_uint8_exact_window_sums(gf, s, mode):
    """uint8 storage: the window sums of J, J^2, P, J P are exact integers (compared bit for bit with the
    oracle's sums of the subsampled values, which are exact in FP64), and q matches the oracle run on the
    dequantised values."""
    H, W, C, r, eps = 240, 328, 3, 16, 1e-3
    I8 = synth.quantize_u8(synth.make_scene(H, W, seed=9))
    p8 = synth.quantize_u8(synth.rgb_noisy_input(I8 / 255.0, seed=10))
    h, w, rl = gf.lowres_geometry(H, W, s, r)
    k = 4 if (mode == 1 and s > 1 and s % 2 == 0) else 1
    st = torch.zeros((1, C, 4, h, w), dtype=torch.int32, device="cuda")
    q = gf.fast_guided_filter(torch.from_numpy(I8).cuda(), torch.from_numpy(p8).cuda(), r, eps, s,
                              MODE_NAMES[mode], stats_out=st)
    torch.cuda.synchronize()
    got = st.cpu().numpy().view(np.uint32).astype(np.int64)
    J = k * oracle.subsample(I8.astype(np.float64), s, mode)
    assert np.all(J == np.round(J))
    for c in range(C):
        P = k * oracle.subsample(p8[c].astype(np.float64), s, mode)
        ref = [oracle.box_sum(J, rl), oracle.box_sum(J * J, rl), oracle.box_sum(P, rl), oracle.box_sum(J * P, rl)]
        for qi in range(4):
            np.testing.assert_array_equal(got[0, c, qi], ref[qi].astype(np.int64))
    ref_q = oracle_q(I8 / 255.0, p8 / 255.0, r, eps, s, mode)
    assert max_abs(q.cpu(), ref_q) <= TOL_F32


def test_lowres_p_box_depthwise(gf):
    """Trainable-layer shape: 3-channel guide guiding each channel of a low-res p (box subsample, r' = 2)."""
    I, p = synth.trainable_layer_batch(batch=2, channels=3, size=128, s=4)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), 0, 1e-2, 4, "box",
                              r_low=2, p_lowres=True)
    torch.cuda.synchronize()
    ref = oracle_q(I, p, 0, 1e-2, 4, 2, r_low=2, p_lowres=True)
    assert max_abs(q.cpu(), ref) <= TOL_F32


def test_host_buffers_match_device_call(gf):
    I = _rand((1, 1, 90, 130), 11)
    p = _rand((1, 3, 90, 130), 12)
    q_dev = _run(gf, I, p, 8, 1e-2, 4, 1)
    q_host = gf.fast_guided_filter_host(torch.from_numpy(I), torch.from_numpy(p), 8, 1e-2, 4, "bilinear").numpy()
    np.testing.assert_array_equal(q_host, q_dev)


@pytest.mark.parametrize("N,CI,C,H,W,s,mode,dtype,pinned", [
    (1, 1, 3, 1100, 900, 4, 1, torch.float32, False),   # ragged last strip, pageable host memory
    (1, 1, 3, 1100, 904, 4, 1, torch.float32, True),    # pinned: the copies overlap
    (2, 3, 3, 600, 700, 4, 2, torch.float16, True),     # batch, depthwise guide, FP16 storage, box
    (1, 1, 3, 1200, 1000, 8, 0, torch.uint8, True),     # uint8, s = 8 nearest
    (1, 1, 3, 1102, 900, 3, 1, torch.float32, True),    # odd s: rows 1, 2 of each block; partial last block
    (1, 1, 1, 2050, 1200, 8, 0, torch.float32, True),   # nearest s = 8, partial last block (rows clamped)
])
def test_host_pipeline_matches_device_call(gf, N, CI, C, H, W, s, mode, dtype, pinned):
    """Large host calls run as a strip pipeline (uploads, row-range filters and downloads overlapping on
    three streams, only the sampled rows of p uploaded for nearest / bilinear at s >= 3); every strip equals
    the same rows of the one-piece device call up to FP32 rounding order and the FP64 oracle within the
    path's tolerance."""
    ys = gf.host_strips(H, W, C, s, MODE_NAMES[mode], batch=N, guide_channels=CI, dtype=dtype)
    assert ys is not None and len(ys) >= 3
    I = _rand((N, CI, H, W), 21)
    p = _rand((N, C, H, W), 22)
    if dtype == torch.uint8:
        Iq, pq = (np.round(I * 255.0).astype(np.uint8), np.round(p * 255.0).astype(np.uint8))
        I_t, p_t = torch.from_numpy(Iq), torch.from_numpy(pq)
        I_ref, p_ref = Iq / 255.0, pq / 255.0
        tol = TOL_F32
    elif dtype == torch.float16:
        I_t, p_t = torch.from_numpy(I).half(), torch.from_numpy(p).half()
        I_ref, p_ref = I_t.double().numpy(), p_t.double().numpy()
        tol = TOL_F16
    else:
        I_t, p_t = torch.from_numpy(I), torch.from_numpy(p)
        I_ref, p_ref = I.astype(np.float64), p.astype(np.float64)
        tol = TOL_F32
    if pinned:
        I_t, p_t = I_t.pin_memory(), p_t.pin_memory()
    ctx = gf.Context(0)
    q_host = gf.fast_guided_filter_host(I_t, p_t, 16, 1e-3, s, MODE_NAMES[mode], ctx=ctx)
    q_host2 = gf.fast_guided_filter_host(I_t, p_t, 16, 1e-3, s, MODE_NAMES[mode], ctx=ctx)  # reused streams
    q_dev = gf.fast_guided_filter(I_t.cuda(), p_t.cuda(), 16, 1e-3, s, MODE_NAMES[mode], ctx=ctx)
    torch.cuda.synchronize()
    q_host, q_host2, q_dev = q_host.float().numpy(), q_host2.float().numpy(), q_dev.float().cpu().numpy()
    np.testing.assert_array_equal(q_host, q_host2)
    assert max_abs(q_host, q_dev) <= (2e-3 if dtype == torch.float16 else 2e-5)
    ref = oracle_q(I_ref, p_ref, 16, 1e-3, s, mode)
    assert max_abs(q_host, ref) <= tol


def test_caller_workspace(gf):
    import ctypes
    I = _rand((1, 1, 70, 90), 13)
    p = _rand((1, 2, 70, 90), 14)
    o = gf.opts_init()
    nbytes = ctypes.c_size_t()
    gf.binding.check(gf.load_library().gf_workspace_size(70, 90, 2, 4, ctypes.byref(o), ctypes.byref(nbytes)))
    ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
    q1 = _run(gf, I, p, 8, 1e-2, 4, 1, workspace=ws)
    q2 = _run(gf, I, p, 8, 1e-2, 4, 1)
    np.testing.assert_array_equal(q1, q2)
    with pytest.raises(gf.GFError) as ei:
        _run(gf, I, p, 8, 1e-2, 4, 1, workspace=ws[:16])
    assert ei.value.status == gf.GF_EINVAL


def test_invalid_arguments_rejected(gf):
    I = torch.rand(1, 2, 16, 16, device="cuda")
    p = torch.rand(1, 3, 16, 16, device="cuda")
    with pytest.raises(gf.GFError) as ei:
        gf.fast_guided_filter(I, p, 2, 1e-2, 2)        # 2 guide channels for 3 input channels
    assert ei.value.status == gf.GF_EINVAL
    with pytest.raises(gf.GFError):
        gf.fast_guided_filter(I[:, :1], p, 2, -1.0, 2)  # eps < 0
    I8 = torch.zeros(16, 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(gf.GFError):
        gf.fast_guided_filter(I8, I8, 2, 1e-2, 2, "box")  # uint8 supports nearest / bilinear only


def test_empty_input_returns_empty(gf):
    I = torch.rand(1, 1, 0, 16, device="cuda")
    p = torch.rand(1, 3, 0, 16, device="cuda")
    q = gf.fast_guided_filter(I, p, 2, 1e-2, 2)
    assert q.shape == (1, 3, 0, 16)


def test_kernel_events_recorded(gf):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * gf.GF_MAX_STAGES)]
    I = _rand((1, 1, 256, 256), 15)
    _run(gf, I, I, 8, 1e-2, 4, 1, kernel_events=ev, fused=-1)
    for k in range(4):  # subsample, statistics + coefficients, box means of a and b, upsample + output
        assert ev[2 * k].elapsed_time(ev[2 * k + 1]) >= 0.0
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(2 * gf.GF_MAX_STAGES)]
    _run(gf, I, I, 8, 1e-2, 4, 1, kernel_events=ev1, fused=1)  # one kernel
    assert ev1[0].elapsed_time(ev1[1]) >= 0.0


def test_precision_variants_at_12mp(gf, scene12mp):
    """Storage precision at 12 MP (r = 16, eps = 1e-3, s = 4 bilinear): FP32, FP16 storage (FP32 arithmetic)
    and uint8 storage (exact integer window sums), each against the FP64 oracle run on the values actually
    stored.  Prints max-abs / RMS per variant (and the FP16 / uint8 distance from the FP32-input result)."""
    I, p = scene12mp
    r, eps, s = 16, 1e-3, 4
    ref32 = oracle_q(I, p, r, eps, s, 1)
    report = {}
    q32 = _run(gf, I, p, r, eps, s, 1)
    report["f32"] = (max_abs(q32, ref32), float(np.sqrt(np.mean((q32 - ref32) ** 2))))
    I16, p16 = synth.to_f16_values(I), synth.to_f16_values(p)
    q16 = gf.fast_guided_filter(torch.from_numpy(I16).cuda(), torch.from_numpy(p16).cuda(), r, eps, s, "bilinear")
    torch.cuda.synchronize()
    q16 = q16.float().cpu().numpy().astype(np.float64)
    ref16 = oracle_q(I16.astype(np.float64), p16.astype(np.float64), r, eps, s, 1)
    report["f16"] = (max_abs(q16, ref16), float(np.sqrt(np.mean((q16 - ref16) ** 2))), max_abs(q16, ref32))
    I8, p8 = synth.quantize_u8(I), synth.quantize_u8(p)
    q8 = gf.fast_guided_filter(torch.from_numpy(I8).cuda(), torch.from_numpy(p8).cuda(), r, eps, s, "bilinear")
    torch.cuda.synchronize()
    q8 = q8.cpu().numpy().astype(np.float64)
    ref8 = oracle_q(I8 / 255.0, p8 / 255.0, r, eps, s, 1)
    report["u8"] = (max_abs(q8, ref8), float(np.sqrt(np.mean((q8 - ref8) ** 2))), max_abs(q8, ref32))
    print("precision report (max-abs, rms[, max-abs vs FP32-input oracle]):", report)
    assert report["f32"][0] <= TOL_F32
    assert report["f16"][0] <= TOL_F16
    assert report["u8"][0] <= TOL_F32


RATIONAL_CASES = [  # (N, CI, C, H, W, r, eps, s, mode, dtype)
    (1, 1, 3, 300, 704, 16, 1e-3, Fraction(5, 2), 1, torch.float32),
    (1, 1, 1, 61, 43, 6, 1e-3, Fraction(3, 2), 0, torch.float32),
    (1, 1, 2, 203, 408, 16, 1e-3, Fraction(7, 4), 3, torch.float32),
    (2, 3, 3, 97, 130, 8, 1e-2, Fraction(4, 3), 1, torch.float32),   # not a binary fraction; depthwise, batch
    (1, 1, 3, 480, 640, 12, 1e-2, Fraction(9, 4), 1, torch.float16),
    (1, 1, 1, 5, 3, 4, 1e-2, Fraction(5, 2), 1, torch.float32),       # tiny, every tap clamped
    (1, 1, 3, 1000, 1500, 20, 1e-3, Fraction(10, 3), 1, torch.float32),
]


@pytest.mark.parametrize("case", RATIONAL_CASES, ids=lambda c: "%dx%d_s%s_m%d_%s" % (c[3], c[4], str(c[7]).replace("/", "o"),
                                                                                       c[8], str(c[9]).split(".")[-1]))
@pytest.mark.parametrize("fused", [-1, 0], ids=["chain", "auto"])
def test_non_integer_ratio_parity(gf, case, fused):
    N, CI, C, H, W, r, eps, s, mode, dtype = case
    I = _rand((N, CI, H, W), 11 + H)
    p = _rand((N, C, H, W), 12 + W)
    if dtype == torch.float16:
        I, p = I.astype(np.float16), p.astype(np.float16)
    q = gf.fast_guided_filter(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(), r, eps, s, MODE_NAMES[mode],
                              fused=fused)
    torch.cuda.synchronize()
    ref = oracle_q(I.astype(np.float64), p.astype(np.float64), r, eps, s, mode)
    err = max_abs(q.float().cpu().numpy(), ref)
    assert err <= (TOL_F16 if dtype == torch.float16 else TOL_F32), "max-abs error %.3g" % err


def test_non_integer_ratio_argument_checks(gf):
    I = torch.rand(1, 1, 64, 64, device="cuda")
    for mode in ("box",):
        with pytest.raises(gf.GFError):
            gf.fast_guided_filter(I, I, 8, 1e-2, Fraction(5, 2), mode)
    with pytest.raises(gf.GFError):
        gf.fast_guided_filter((I * 255).to(torch.uint8), (I * 255).to(torch.uint8), 8, 1e-2, Fraction(5, 2))
    with pytest.raises(gf.GFError):
        gf.fast_guided_filter_backward(I, I, I, 8, 1e-2, Fraction(5, 2))
    # an integer written as a fraction is the integer ratio
    a = gf.fast_guided_filter(I, I, 8, 1e-2, Fraction(8, 2))
    b = gf.fast_guided_filter(I, I, 8, 1e-2, 4)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("s,mode", [(2, "bilinear"), (4, "bilinear"), (8, "bilinear"), (4, "nearest")])
@pytest.mark.parametrize("dtype", [torch.float16, torch.uint8])
def test_vector_subsample_matches_generic_path(gf, s, mode, dtype):
    """FP16 / uint8 storage: 16-byte aligned planes take the vector subsample, the same data one element off
    the alignment takes the generic one; the results agree (uint8: the same exact integer window sums)."""
    H, W, C = 256, 512, 3
    I = torch.from_numpy(synth.make_scene(H, W, seed=31)).cuda()[None, None]
    p = torch.from_numpy(synth.rgb_noisy_input(synth.make_scene(H, W, seed=31), seed=32)).cuda()[None]
    if dtype == torch.uint8:
        I, p = (I * 255).round().to(dtype), (p * 255).round().to(dtype)
    else:
        I, p = I.to(dtype), p.to(dtype)

    def shifted(t):  # the same values at an address one element past a 16-byte boundary
        buf = torch.empty(t.numel() + 16, dtype=t.dtype, device="cuda")
        v = buf[1:1 + t.numel()].view(t.shape)
        v.copy_(t)
        return v

    st_a = torch.empty((1, C, 4, -(-H // s), -(-W // s)), dtype=torch.int32 if dtype == torch.uint8 else torch.float32,
                       device="cuda")
    st_b = torch.empty_like(st_a)
    qa = gf.fast_guided_filter(I, p, 4 * s, 1e-2, s, mode, stats_out=st_a)
    qb = gf.fast_guided_filter(shifted(I), shifted(p), 4 * s, 1e-2, s, mode, stats_out=st_b)
    torch.cuda.synchronize()
    assert torch.equal(st_a, st_b)  # the subsampled values, hence every window sum, are identical
    # the two output kernels round in a different order; FP16 q may differ by one unit in the last place
    assert float((qa.float() - qb.float()).abs().max()) <= (1e-3 if dtype == torch.float16 else 1e-6)
