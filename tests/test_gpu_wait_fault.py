"""A bounded wait inside a kernel that runs out: reported, not hidden, and the GPU stays usable.

The TMA-fed output kernel (Algorithm 2's upsample and output, s = 4 and 8) hands each stage of its ring from a
producer lane to the consumer warps through mbarriers, and every wait is bounded.  gf_opts.test_wait_fault
makes the producer leave the first stage unfilled (a flag that nothing sets) and shortens those waits to 256
polls: the consumers' first wait runs out, the kernel records the timeout and returns with q incomplete -- no
trap, no endless loop, no GPU fault.  Checked: the device-wide fault bits, gf_filter_host returning GF_EWAIT,
and the next ordinary call on the same GPU matching the FP64 oracle with no fault recorded.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import TOL_F32, max_abs, oracle_q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    gf.kernel_faults(clear=True)
    return gf


def _inputs(H, W, C, seed):
    g = np.random.default_rng(seed)
    return g.uniform(0, 1, (1, 1, H, W)).astype(np.float32), g.uniform(0, 1, (1, C, H, W)).astype(np.float32)


def test_device_call_records_the_timeout_and_the_next_call_is_green(gf):
    I, p = _inputs(256, 1024, 3, 1)
    Id, pd = torch.from_numpy(I).cuda(), torch.from_numpy(p).cuda()
    q = torch.full((1, 3, 256, 1024), -1.0, device="cuda")
    gf.fast_guided_filter(Id, pd, 16, 1e-3, 4, "bilinear", out=q, fused=-1, test_wait_fault=True)
    torch.cuda.synchronize()
    faults = gf.kernel_faults(clear=True)
    assert faults & 1, "the output kernel's bounded wait should have given up"
    assert bool((q == -1.0).any()), "rows of the skipped stage are left unwritten"
    # the same GPU, the next ordinary call: complete and correct, nothing recorded
    q2 = gf.fast_guided_filter(Id, pd, 16, 1e-3, 4, "bilinear", fused=-1)
    torch.cuda.synchronize()
    assert gf.kernel_faults(clear=True) == 0
    assert max_abs(q2.cpu(), oracle_q(I, p, 16, 1e-3, 4, oracle.SUB_BILINEAR)) <= TOL_F32


def test_host_call_returns_ewait(gf):
    I, p = _inputs(640, 1024, 3, 2)
    with pytest.raises(gf.GFError) as ei:
        gf.fast_guided_filter_host(torch.from_numpy(I), torch.from_numpy(p), 16, 1e-3, 4, "bilinear", fused=-1,
                                   test_wait_fault=True)
    assert ei.value.status == gf.GF_EWAIT
    gf.kernel_faults(clear=True)
    q = gf.fast_guided_filter_host(torch.from_numpy(I), torch.from_numpy(p), 16, 1e-3, 4, "bilinear", fused=-1)
    assert gf.kernel_faults(clear=True) == 0
    assert max_abs(q.numpy(), oracle_q(I, p, 16, 1e-3, 4, oracle.SUB_BILINEAR)) <= TOL_F32
