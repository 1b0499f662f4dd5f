"""GPU parity of the hand-written backward pass (gf_filter_backward) and the autograd layer.

References: the FP64 oracle's adjoint (pinned on CPU to central differences and float64 autograd), a
float64 torch-autograd restatement, and at the full trainable-layer shape (16 x 3 x 1024 x 1024 guide,
16 x 3 x 256 x 256 low-res p, s = 4, r' = 2, eps = 1e-2, box subsample) a random-direction central
difference of the FP64 oracle forward with h = 1e-3.

Tolerance: the gradient runs in FP32 through the divisions by (var + eps); a relative rounding of about
1e-6 in the window sums is amplified by up to ~1/eps on the way to dI and dp, so each gradient is compared
as max|gpu - ref| <= 2e-4 * max|ref| + 1e-6 (for eps >= 1e-3; the directional checks use 1e-3 relative).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import torch_restatement as tr

pytestmark = pytest.mark.gpu

MODE_NAMES = {0: "nearest", 1: "bilinear", 2: "box", 3: "bilinear_aa"}


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _close(got, ref, rel=2e-4, floor=1e-6):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = float(np.max(np.abs(got - ref)))
    bound = rel * float(np.max(np.abs(ref))) + floor
    assert err <= bound, "max-abs error %.3g > %.3g" % (err, bound)


BWD_CASES = [
    # (N, CI, C, H, W, r_low, eps, s, mode, p_lowres)
    (1, 1, 1, 16, 20, 2, 1e-2, 1, 1, False),
    (1, 1, 3, 37, 53, 2, 1e-2, 2, 1, False),
    (2, 3, 3, 64, 64, 2, 1e-2, 4, 2, True),
    (1, 1, 2, 61, 43, 1, 5e-2, 3, 0, False),
    (1, 1, 3, 120, 200, 4, 1e-3, 4, 1, False),
    (1, 1, 1, 50, 70, 20, 1e-2, 1, 1, False),
    (1, 3, 3, 96, 136, 2, 1e-2, 8, 1, False),
    (1, 1, 3, 97, 130, 3, 1e-2, 4, 2, False),
    (1, 1, 1, 1, 9, 1, 1e-2, 2, 1, False),
    (1, 1, 2, 45, 57, 2, 1e-2, 3, 1, False),   # odd s, bilinear: every sample on a pixel (weights 1, 0)
    # vector forms of the full-res kernels (s = 4, 8; H, W multiples of s)
    (1, 1, 2, 64, 96, 2, 1e-2, 4, 0, False),   # nearest
    (2, 1, 3, 48, 64, 1, 1e-2, 8, 2, False),   # box, gray guide, full-res p
    (1, 1, 2, 16, 24, 1, 1e-2, 8, 1, False),   # w = 3: both edge blocks and one inside
    (1, 1, 1, 16, 8, 1, 1e-2, 8, 0, False),    # w = 1: one block at both edges (h = 2: var > 0)
    (1, 1, 2, 280, 260, 2, 1e-2, 4, 1, False), # h = 70, w = 65: several column tiles and row chunks of U^T
    (1, 1, 1, 528, 496, 1, 1e-2, 8, 0, False), # s = 8: h = 66, w = 62
]


@pytest.mark.parametrize("case", BWD_CASES, ids=lambda c: "N%dCI%dC%d_%dx%d_r%d_s%d_m%d_pl%d" % (c[0], c[1], c[2], c[3], c[4], c[5], c[7], c[8], c[9]))
def test_backward_matches_oracle(gf, case):
    N, CI, C, H, W, rl, eps, s, mode, p_lowres = case
    rng = np.random.default_rng(H * 31 + W)
    h, w = oracle.lowres_shape(H, W, s)
    I = rng.uniform(0, 1, (N, CI, H, W)).astype(np.float32)
    p = rng.uniform(0, 1, (N, C, h, w) if p_lowres else (N, C, H, W)).astype(np.float32)
    Wt = rng.uniform(-1, 1, (N, C, H, W)).astype(np.float32)
    dI, dp, deps = gf.fast_guided_filter_backward(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(),
                                                  torch.from_numpy(Wt).cuda(), 0, eps, s, MODE_NAMES[mode], r_low=rl,
                                                  p_lowres=p_lowres)
    torch.cuda.synchronize()
    rdI, rdp, rdeps = oracle.fast_guided_filter_backward(I, p, Wt, 0, eps, s, mode, r_low=rl, p_lowres=p_lowres)
    _close(dI.cpu(), rdI)
    _close(dp.cpu(), rdp)
    assert float(deps) == pytest.approx(rdeps, rel=1e-3, abs=1e-5)


def test_backward_matches_float64_autograd(gf):
    rng = np.random.default_rng(5)
    N, C, H, W, rl, eps, s = 2, 3, 96, 128, 3, 1e-2, 4
    I = rng.uniform(0, 1, (N, 1, H, W)).astype(np.float32)
    p = rng.uniform(0, 1, (N, C, H, W)).astype(np.float32)
    Wt = rng.uniform(-1, 1, (N, C, H, W)).astype(np.float32)
    dI, dp, deps = gf.fast_guided_filter_backward(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(),
                                                  torch.from_numpy(Wt).cuda(), 0, eps, s, "bilinear", r_low=rl)
    tI = torch.tensor(I, dtype=torch.float64, requires_grad=True)
    tp = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    te = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    (tr.fast_guided_filter(tI, tp, rl, te, s, 1) * torch.from_numpy(Wt).double()).sum().backward()
    _close(dI.cpu(), tI.grad)
    _close(dp.cpu(), tp.grad)
    assert float(deps) == pytest.approx(te.grad.item(), rel=1e-3)


@pytest.fixture(scope="module")
def layer_batch():
    I, p = synth.trainable_layer_batch(batch=16, channels=3, size=1024, s=4)
    Wt = np.random.default_rng(99).uniform(-1, 1, I.shape).astype(np.float32)
    return I, p, Wt


def test_trainable_layer_full_shape_directional_derivative(gf, layer_batch):
    """16 x 3 x 1024^2 guide, low-res p 16 x 3 x 256^2, s = 4, r' = 2, eps = 1e-2, box subsample:
    <dL/dI, vI> + <dL/dp, vp> + dL/deps * ve from the GPU against a central difference of the FP64 oracle
    forward along the same random direction (h = 1e-3)."""
    I, p, Wt = layer_batch
    eps, hstep = 1e-2, 1e-3
    dI, dp, deps = gf.fast_guided_filter_backward(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(),
                                                  torch.from_numpy(Wt).cuda(), 0, eps, 4, "box", r_low=2, p_lowres=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    vI = rng.standard_normal(I.shape)
    vp = rng.standard_normal(p.shape)
    ve = 1.0
    I64, p64, W64 = I.astype(np.float64), p.astype(np.float64), Wt.astype(np.float64)

    def loss(t):
        q = oracle.fast_guided_filter(I64 + t * vI, p64 + t * vp, 0, eps + t * ve, 4, oracle.SUB_BOX, r_low=2,
                                      p_lowres=True)
        return float(np.sum(q * W64))

    fd = (loss(hstep) - loss(-hstep)) / (2 * hstep)
    an = float(np.sum(dI.cpu().numpy().astype(np.float64) * vI) + np.sum(dp.cpu().numpy().astype(np.float64) * vp)
               + float(deps) * ve)
    assert an == pytest.approx(fd, rel=1e-3)


def test_trainable_layer_full_shape_elementwise_sample(gf, layer_batch):
    """Two images of the full batch, every gradient element against the FP64 oracle adjoint."""
    I, p, Wt = layer_batch
    eps = 1e-2
    dI, dp, deps = gf.fast_guided_filter_backward(torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda(),
                                                  torch.from_numpy(Wt).cuda(), 0, eps, 4, "box", r_low=2, p_lowres=True)
    torch.cuda.synchronize()
    for b in (0, 15):
        rdI, rdp, _ = oracle.fast_guided_filter_backward(I[b:b + 1], p[b:b + 1], Wt[b:b + 1], 0, eps, 4, oracle.SUB_BOX,
                                                        r_low=2, p_lowres=True)
        _close(dI[b:b + 1].cpu(), rdI)
        _close(dp[b:b + 1].cpu(), rdp)


def test_autograd_layer(gf):
    rng = np.random.default_rng(11)
    I = torch.from_numpy(rng.uniform(0, 1, (2, 3, 64, 64)).astype(np.float32)).cuda().requires_grad_(True)
    p = torch.from_numpy(rng.uniform(0, 1, (2, 3, 16, 16)).astype(np.float32)).cuda().requires_grad_(True)
    Wt = torch.from_numpy(rng.uniform(-1, 1, (2, 3, 64, 64)).astype(np.float32)).cuda()
    layer = gf.FastGuidedFilter(r=0, eps=1e-2, s=4, mode="box", r_low=2, p_lowres=True, learn_eps=True).cuda()
    (layer(I, p) * Wt).sum().backward()
    dI, dp, deps = gf.fast_guided_filter_backward(I.detach(), p.detach(), Wt, 0, 1e-2, 4, "box", r_low=2, p_lowres=True)
    torch.cuda.synchronize()
    assert torch.equal(I.grad, dI) and torch.equal(p.grad, dp)
    assert layer.eps.grad is not None and float(layer.eps.grad) == pytest.approx(float(deps), rel=1e-6)
    # a 2% step of eps against its gradient lowers the loss by about the first-order amount
    with torch.no_grad():
        l0 = float((layer(I, p) * Wt).sum(dtype=torch.float64))
        step = -0.02 * float(layer.eps) * float(layer.eps.grad.sign())
        layer.eps += step
        l1 = float((layer(I, p) * Wt).sum(dtype=torch.float64))
    assert l1 < l0
    assert (l1 - l0) == pytest.approx(step * float(deps), rel=0.2)


def test_backward_is_deterministic(gf):
    rng = np.random.default_rng(12)
    I = torch.from_numpy(rng.uniform(0, 1, (1, 1, 200, 300)).astype(np.float32)).cuda()
    p = torch.from_numpy(rng.uniform(0, 1, (1, 3, 200, 300)).astype(np.float32)).cuda()
    g = torch.from_numpy(rng.uniform(-1, 1, (1, 3, 200, 300)).astype(np.float32)).cuda()
    a = gf.fast_guided_filter_backward(I, p, g, 8, 1e-2, 4, "bilinear")
    b = gf.fast_guided_filter_backward(I, p, g, 8, 1e-2, 4, "bilinear")
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_antialiased_subsample_is_forward_only(gf):
    I = torch.rand(1, 1, 32, 32, device="cuda")
    with pytest.raises(gf.GFError) as ei:
        gf.fast_guided_filter_backward(I, I, I, 4, 1e-2, 4, "bilinear_aa")
    assert ei.value.status == gf.GF_EINVAL


@pytest.mark.parametrize("case", [
    (1, 1, 3, 120, 200, 4, 1e-3, 4, 1, False),   # gray guide, bilinear
    (2, 3, 3, 64, 64, 2, 1e-2, 4, 2, True),      # depthwise guide, box, low-res p
    (1, 1, 2, 61, 43, 1, 5e-2, 3, 0, False),     # odd s, nearest, ragged
], ids=lambda c: "N%dCI%dC%d_%dx%d_s%d_m%d" % (c[0], c[1], c[2], c[3], c[4], c[7], c[8]))
def test_saved_forward_equals_recomputation(gf, case):
    """gf_opts.saved_forward: the forward keeps its low-res planes in the backward's workspace and the backward
    skips recomputing them.  q and every gradient equal those of the plain forward and the recomputing
    backward bit for bit (the same kernels compute the same planes)."""
    N, CI, C, H, W, rl, eps, s, mode, p_lowres = case
    rng = np.random.default_rng(7 * H + W)
    h, w = oracle.lowres_shape(H, W, s)
    I = torch.from_numpy(rng.uniform(0, 1, (N, CI, H, W)).astype(np.float32)).cuda()
    p = torch.from_numpy(rng.uniform(0, 1, (N, C, h, w) if p_lowres else (N, C, H, W)).astype(np.float32)).cuda()
    g = torch.from_numpy(rng.uniform(-1, 1, (N, C, H, W)).astype(np.float32)).cuda()
    kw = dict(r_low=rl, p_lowres=p_lowres)
    q_plain = gf.fast_guided_filter(I, p, 0, eps, s, MODE_NAMES[mode], fused=-1, **kw)
    ws = torch.empty(gf.backward_workspace_size(H, W, C, s, batch=N, guide_channels=CI, **kw), dtype=torch.uint8,
                     device="cuda")
    q_saved = gf.fast_guided_filter(I, p, 0, eps, s, MODE_NAMES[mode], workspace=ws, saved_forward=True, **kw)
    ref = gf.fast_guided_filter_backward(I, p, g, 0, eps, s, MODE_NAMES[mode], **kw)
    got = gf.fast_guided_filter_backward(I, p, g, 0, eps, s, MODE_NAMES[mode], workspace=ws, saved_forward=True, **kw)
    got2 = gf.fast_guided_filter_backward(I, p, g, 0, eps, s, MODE_NAMES[mode], workspace=ws, saved_forward=True, **kw)
    torch.cuda.synchronize()
    assert torch.equal(q_saved, q_plain)
    for a, b, c in zip(got, ref, got2):
        assert torch.equal(a, b)
        assert torch.equal(c, b)  # the backward leaves the saved planes as they were
    with pytest.raises(gf.GFError) as ei:  # the saving forward needs the workspace
        gf.fast_guided_filter(I, p, 0, eps, s, MODE_NAMES[mode], saved_forward=True, **kw)
    assert ei.value.status == gf.GF_EINVAL
