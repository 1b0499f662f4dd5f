"""gf_filter_noalloc: the forward filter for callers that cannot allocate device memory.

Such callers -- a plugin whose host application owns all device memory, or code that must not enter the
allocator on a latency-critical path -- get the filter's scratch from a fixed array inside the library
instead of cudaMalloc.  This test calls that entry point through the C ABI twice in a row with the
multi-kernel chain forced (gf_opts.fused = -1, so both calls keep their low-res planes in the shared
array): first a large problem, then a smaller one, so that the second call starts from the first call's
leftover planes and any plane it failed to rewrite would show.  Each result is compared with the FP64
oracle and with the ordinary gf_filter entry point at the parity tolerance of the other GPU tests.  It
also checks that a call needing more scratch than the array holds is refused with GF_EINVAL.  The file
sorts last so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-4  # max-abs tolerance of the FP32 parity tests


def _inputs(N, C, H, W, seed):
    g = torch.Generator().manual_seed(seed)
    I = torch.rand((N, 1, H, W), generator=g)
    p = torch.rand((N, C, H, W), generator=g)
    return I, p


def _noalloc(lib, gf, I, p, r, eps, s, mode):
    N, _, H, W = I.shape
    C = p.shape[1]
    q = torch.full((N, C, H, W), float("nan"), device="cuda")
    o = gf.opts_init()
    o.batch = N
    o.fused = -1  # the chain: every low-res plane lives in the static scratch
    st = torch.cuda.current_stream()
    status = lib.gf_filter_noalloc(ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                   ctypes.c_void_p(q.data_ptr()), H, W, C, r, eps, s, gf.MODES[mode],
                                   ctypes.byref(o), ctypes.c_void_p(st.cuda_stream))
    assert status == gf.GF_OK, lib.gf_last_error()
    return q


def test_noalloc_matches_oracle_and_gf_filter_on_two_calls_in_a_row(cuda_device):
    import paper_1505_00996_gb300 as gf
    lib = gf.load_library()
    problems = [  # (N, C, H, W, r, eps, s, mode): large first, so the second call reuses its leftovers
        (1, 3, 600, 800, 16, 1e-3, 4, "bilinear"),
        (2, 1, 241, 333, 8, 1e-2, 2, "nearest"),
    ]
    for k, (N, C, H, W, r, eps, s, mode) in enumerate(problems):
        I, p = _inputs(N, C, H, W, seed=k)
        Id, pd = I.cuda(), p.cuda()
        q = _noalloc(lib, gf, Id, pd, r, eps, s, mode)
        q_ref = gf.fast_guided_filter(Id, pd, r, eps, s, mode, fused=-1)
        torch.cuda.synchronize()
        assert torch.isfinite(q).all()
        q_or = oracle.fast_guided_filter(I.numpy().astype(np.float64), p.numpy().astype(np.float64), r, eps, s,
                                         gf.MODES[mode])
        err_or = float(np.max(np.abs(q.cpu().numpy().astype(np.float64) - q_or)))
        err_gf = float((q - q_ref).abs().max())
        assert err_or <= TOL, "call %d: max-abs error against the oracle %.3g" % (k, err_or)
        assert err_gf <= TOL, "call %d: max-abs difference from gf_filter %.3g" % (k, err_gf)


def test_noalloc_refuses_calls_beyond_its_scratch(cuda_device):
    import paper_1505_00996_gb300 as gf
    lib = gf.load_library()
    # s = 1 at 12 MP with 3 channels needs far more than the 64 MiB static scratch
    H, W, C = 3000, 4000, 3
    I = torch.zeros((1, 1, 8, 8), device="cuda")  # never read: the size check comes first
    o = gf.opts_init()
    status = lib.gf_filter_noalloc(ctypes.c_void_p(I.data_ptr()), ctypes.c_void_p(I.data_ptr()),
                                   ctypes.c_void_p(I.data_ptr()), H, W, C, 16, 1e-3, 1, gf.GF_SUB_BILINEAR,
                                   ctypes.byref(o), None)
    assert status == gf.GF_EINVAL
    assert b"static scratch" in lib.gf_last_error()
