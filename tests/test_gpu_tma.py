"""The TMA-fed output kernel (gf_tma.cu): the guide rows reach shared memory as cp.async.bulk.tensor tiles
through an mbarrier producer/consumer ring instead of per-thread copies.  The arithmetic is the same as the
per-thread-copy kernel, so both must give bit-identical q; the environment variable GF_NO_TMA selects the
per-thread-copy kernel for the comparison.  Also: no bounded wait gave up (gf_kernel_faults), and the path
holds at the 12 MP workload, for FP16 / uint8 storage, depthwise guides, s = 8, ragged widths and strips.
"""
import os

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import TOL_F32, max_abs, oracle_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    gf.kernel_faults(clear=True)
    return gf


def _both(gf, *args, **kw):
    q_tma = gf.fast_guided_filter(*args, **kw)
    torch.cuda.synchronize()
    os.environ["GF_NO_TMA"] = "1"
    try:
        q_ref = gf.fast_guided_filter(*args, **kw)
        torch.cuda.synchronize()
    finally:
        del os.environ["GF_NO_TMA"]
    return q_tma, q_ref


CASES = [  # (N, CI, C, H, W, r, s, dtype)
    (1, 1, 3, 3000, 4000, 16, 4, torch.float32),   # the 12 MP workload
    (1, 1, 3, 1000, 1504, 16, 8, torch.float32),
    (2, 3, 3, 517, 1032, 8, 4, torch.float32),     # depthwise guide, batch, ragged last band
    (1, 1, 2, 700, 904, 8, 4, torch.float16),
    (1, 1, 1, 640, 1024, 8, 8, torch.uint8),
    (1, 1, 3, 33, 36, 4, 4, torch.float32),        # one partial band
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%dCI%dC%d_%dx%d_s%d_%s" % (c[0], c[1], c[2], c[3], c[4], c[6],
                                                                                  str(c[7]).split(".")[-1]))
def test_tma_output_equals_per_thread_copies(gf, case):
    N, CI, C, H, W, r, s, dtype = case
    g = np.random.default_rng(H + W)
    I = g.uniform(0, 1, (N, CI, H, W)).astype(np.float32)
    p = g.uniform(0, 1, (N, C, H, W)).astype(np.float32)
    It, pt = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    if dtype == torch.uint8:
        It, pt = (It * 255).round().to(dtype), (pt * 255).round().to(dtype)
    else:
        It, pt = It.to(dtype), pt.to(dtype)
    q_tma, q_ref = _both(gf, It, pt, r, 1e-2, s, "bilinear", fused=-1)
    assert torch.equal(q_tma, q_ref)
    assert gf.kernel_faults(clear=True) == 0
    if H * W <= 1_000_000 and dtype == torch.float32:
        assert max_abs(q_tma.cpu().numpy(), oracle_q(I, p, r, 1e-2, s, 1)) <= TOL_F32


def test_tma_output_in_strips(gf):
    I = torch.from_numpy(synth.make_scene(800, 1024, seed=3)).cuda()[None, None]
    p = I.repeat(1, 3, 1, 1).contiguous()
    whole = gf.fast_guided_filter(I, p, 16, 1e-3, 4, "bilinear", fused=-1)
    q = torch.full_like(whole, float("nan"))
    for rows in gf.row_strips(800, 3):
        gf.fast_guided_filter(I, p, 16, 1e-3, 4, "bilinear", out=q, rows=rows, fused=-1)
    torch.cuda.synchronize()
    assert not torch.isnan(q).any()
    assert float((q - whole).abs().max()) <= 2 * TOL_F32
    assert gf.kernel_faults(clear=True) == 0
