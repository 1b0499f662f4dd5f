"""Serving loop (gf_submit / gf_poll / gf_cancel) on the GPU.

Checks: a mixed batch of requests (sizes, radii, ratios, channel counts, FP16 and FP32 storage) gives, for
every request, exactly the result of running it alone through gf_filter, while requests overlap on the
device, with direct launches, per-bucket graphs and tile-queue launches of several small requests; admission never exceeds the HBM budget or the slot count; a request that can never fit is
refused; held requests report pending / time out and can be cancelled; an injected launch failure fails
only its own request; and a context with queued work shuts down cleanly.
"""
import ctypes
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import TOL_F16, max_abs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf(cuda_device):
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    return gf


def _make(H, W, C, dtype, seed):
    I = synth.make_scene(H, W, seed=seed)
    p = synth.rgb_noisy_input(I, seed=seed + 1, channels=C)
    It = torch.from_numpy(I).to(dtype).cuda()
    pt = torch.from_numpy(p).to(dtype).cuda()
    return It, pt


MIX = [  # (H, W, C, r, eps, s, mode, dtype)
    (480, 640, 3, 3, 1e-4, 4, "bilinear", torch.float16),
    (1080, 1920, 1, 8, 1e-2, 8, "bilinear", torch.float16),
    (700, 700, 3, 4, 1e-2, 4, "nearest", torch.float16),
    (1200, 1600, 3, 6, 1e-4, 8, "bilinear", torch.float16),
    (333, 517, 1, 2, 1e-2, 4, "bilinear", torch.float32),
    (900, 1600, 3, 7, 1e-2, 4, "bilinear", torch.float16),
    (256, 256, 3, 16, 1e-3, 1, "bilinear", torch.float32),
    (1500, 2000, 1, 8, 1e-4, 4, "box", torch.float16),
    (611, 409, 3, 5, 1e-2, 8, "nearest", torch.float32),
    (2000, 2000, 3, 8, 1e-2, 4, "bilinear", torch.float16),
    (100, 3000, 1, 12, 1e-4, 8, "bilinear", torch.float16),
    (768, 1024, 3, 4, 1e-2, 4, "bilinear", torch.float16),
]


@pytest.mark.parametrize("graphs,tile_queue", [(True, False), (False, False), (False, True)],
                         ids=["graphs", "direct", "tile_queue"])
def test_mixed_requests_equal_their_solo_results(gf, graphs, tile_queue):
    """Every request of the mix equals its solo gf_filter result bit for bit, with the per-bucket graphs (the
    mix runs twice, so the second pass replays updated graphs), with direct launches, and with the tile queue
    (neighbouring single-kernel requests in one launch)."""
    inputs = [_make(H, W, C, dt, 100 + k) for k, (H, W, C, r, e, s, m, dt) in enumerate(MIX)]
    refs = []
    for (I, p), (H, W, C, r, e, s, m, dt) in zip(inputs, MIX):
        refs.append(gf.fast_guided_filter(I, p, r, e, s, m))
    torch.cuda.synchronize()
    srv = gf.Server(slots=4, graphs=graphs, tile_queue=tile_queue)
    outs, tickets = [], []
    for rep in range(2):
        for (I, p), (H, W, C, r, e, s, m, dt), ref in zip(inputs, MIX, refs):
            q = torch.full_like(ref, float("nan"))
            outs.append(q)
            tickets.append(srv.submit(I, p, q, r, e, s, m))
    refs = refs + refs
    results = [srv.poll(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert (stats["graph_launches"] > 0) == graphs and stats["launches"] == len(tickets)
    assert tile_queue or stats["queue_launches"] == 0
    assert all(res["status"] == gf.GF_OK for res in results)
    for q, ref in zip(outs, refs):
        assert torch.equal(q, ref)
    # the requests shared the GPU: some admitted request started before another one had finished
    spans = sorted((res["t_admit"], res["t_done"]) for res in results)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    # and one of them against the FP64 oracle at the FP16-storage tolerance
    (I, p), (H, W, C, r, e, s, m, dt) = inputs[0], MIX[0]
    ref64 = oracle.fast_guided_filter(I.float().cpu().numpy().astype(np.float64),
                                      p.float().cpu().numpy().astype(np.float64), r, e, s, oracle.SUB_BILINEAR)
    assert max_abs(outs[0].float().cpu(), ref64) <= TOL_F16


SMALL = [  # single-kernel requests (s > 1, at most 2^20 pixel-channels): (H, W, C, r, eps, s, mode)
    (480, 640, 3, 3, 1e-4, 4, "bilinear"),
    (333, 517, 1, 2, 1e-2, 4, "bilinear"),
    (611, 409, 3, 5, 1e-2, 8, "bilinear"),
    (100, 3000, 1, 12, 1e-4, 8, "bilinear"),
    (256, 256, 3, 4, 1e-3, 2, "bilinear"),
    (97, 131, 1, 1, 1e-2, 4, "bilinear"),
    (512, 512, 3, 8, 1e-2, 4, "bilinear"),
    (300, 700, 2, 6, 1e-4, 4, "bilinear"),
]


@pytest.mark.parametrize("slots", [1, 3])
def test_tile_queue_batches_equal_their_solo_results(gf, slots):
    """Small FP16 requests of mixed sizes, radii, ratios and channel counts queued while admission is held,
    then released: they run in tile-queue launches of several requests each, and every result equals its solo
    gf_filter result bit for bit.  A FP32 request in the middle of the stream starts a batch of its own."""
    reqs = SMALL * 3
    inputs = [_make(H, W, C, torch.float32 if k == 9 else torch.float16, 300 + k)
              for k, (H, W, C, r, e, s, m) in enumerate(reqs)]
    refs = [gf.fast_guided_filter(I, p, r, e, s, m) for (I, p), (H, W, C, r, e, s, m) in zip(inputs, reqs)]
    torch.cuda.synchronize()
    srv = gf.Server(slots=slots)
    srv.pause(True)
    outs = [torch.full_like(ref, float("nan")) for ref in refs]
    tickets = [srv.submit(I, p, q, r, e, s, m) for (I, p), q, (H, W, C, r, e, s, m) in zip(inputs, outs, reqs)]
    srv.pause(False)
    results = [srv.poll(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(res["status"] == gf.GF_OK for res in results)
    assert stats["queue_launches"] >= 2 and stats["queue_requests"] >= len(reqs) - 3
    assert stats["launches"] == len(reqs)
    for q, ref in zip(outs, refs):
        assert torch.equal(q, ref)


def test_admission_respects_budget_and_slots(gf):
    o = gf.opts_init()
    o.dtype_in = gf.GF_F16
    o.dtype_out = gf.GF_F16
    need = ctypes.c_size_t()
    gf.binding.check(gf.load_library().gf_workspace_size(1500, 2000, 3, 4, ctypes.byref(o), ctypes.byref(need)))
    budget = 3 * need.value + 4096
    srv = gf.Server(hbm_budget_bytes=budget, slots=8)
    I, p = _make(1500, 2000, 3, torch.float16, 7)
    qs = [torch.empty((1, 3, 1500, 2000), dtype=torch.float16, device="cuda") for _ in range(16)]
    tickets = [srv.submit(I, p, q, 8, 1e-2, 4, "bilinear") for q in qs]
    peak_scratch, peak_running = 0, 0
    for _ in range(2000):
        st = srv.stats()
        peak_scratch = max(peak_scratch, st["scratch_in_use"])
        peak_running = max(peak_running, st["running"])
        if st["queued"] == 0 and st["running"] == 0:
            break
        time.sleep(0.0005)
    results = [srv.poll(t) for t in tickets]
    srv.close()
    assert all(r["status"] == gf.GF_OK for r in results)
    assert peak_scratch <= budget
    assert peak_running <= 3  # the budget, not the 8 slots, bounds the concurrency here
    ref = gf.fast_guided_filter(I, p, 8, 1e-2, 4, "bilinear")
    torch.cuda.synchronize()
    for q in qs:
        assert torch.equal(q, ref.view_as(q))


def test_request_that_can_never_fit_is_refused(gf):
    srv = gf.Server(hbm_budget_bytes=1 << 20, slots=2)
    I, p = _make(2000, 2000, 3, torch.float32, 8)
    q = torch.empty((1, 3, 2000, 2000), device="cuda")
    with pytest.raises(gf.GFError) as ei:
        srv.submit(I, p, q, 8, 1e-2, 4)
    assert ei.value.status == gf.GF_ENOMEM
    srv.close()


def test_held_requests_pending_timeout_cancel(gf):
    srv = gf.Server(slots=2)
    I, p = _make(300, 400, 3, torch.float32, 9)
    q1 = torch.empty((1, 3, 300, 400), device="cuda")
    q2 = torch.empty_like(q1)
    srv.pause(True)
    t1 = srv.submit(I, p, q1, 4, 1e-2, 4)
    t2 = srv.submit(I, p, q2, 4, 1e-2, 4)
    assert srv.poll_status(t1, 0) == gf.GF_PENDING
    t0 = time.perf_counter()
    assert srv.poll_status(t1, 20000) == gf.GF_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.015
    assert srv.cancel(t2) == gf.GF_OK
    assert srv.stats()["queued"] == 1
    srv.pause(False)
    res = srv.poll(t1)
    assert res["status"] == gf.GF_OK
    assert srv.cancel(t1) == gf.GF_ENOTFOUND  # retired after its result was delivered
    assert srv.poll_status(t2, 0) == gf.GF_ECANCELED
    assert srv.poll_status(t2, 0) == gf.GF_ENOTFOUND
    ref = gf.fast_guided_filter(I, p, 4, 1e-2, 4)
    torch.cuda.synchronize()
    assert torch.equal(q1, ref.view_as(q1))
    srv.close()


def test_injected_launch_failure_fails_only_its_request(gf, monkeypatch):
    monkeypatch.setenv("GF_FAULT", "launch:1")  # read when the context is created
    srv = gf.Server(slots=1)
    I, p = _make(400, 600, 3, torch.float32, 10)
    qs = [torch.empty((1, 3, 400, 600), device="cuda") for _ in range(3)]
    tickets = [srv.submit(I, p, q, 6, 1e-2, 4) for q in qs]
    statuses = [srv.poll(t)["status"] for t in tickets]
    srv.close()
    assert statuses == [gf.GF_OK, gf.GF_ECUDA, gf.GF_OK]
    ref = gf.fast_guided_filter(I, p, 6, 1e-2, 4)
    torch.cuda.synchronize()
    assert torch.equal(qs[0], ref.view_as(qs[0])) and torch.equal(qs[2], ref.view_as(qs[2]))


def test_context_with_queued_work_shuts_down(gf):
    srv = gf.Server(slots=1)
    I, p = _make(200, 300, 1, torch.float32, 11)
    q = torch.empty((1, 1, 200, 300), device="cuda")
    srv.pause(True)
    srv.submit(I, p, q, 4, 1e-2, 4)
    t0 = time.perf_counter()
    srv.close()
    assert time.perf_counter() - t0 < 5.0


def test_inputs_written_on_another_stream_are_waited_for(gf):
    """Inputs still being written when the request is submitted (a long kernel ahead of their copy on the
    producing stream, no synchronize): the request's kernels wait for the event submit records there."""
    H, W, C = 600, 800, 3
    src_I, src_p = _make(H, W, C, torch.float32, 12)
    ref = gf.fast_guided_filter(src_I, src_p, 8, 1e-2, 4, "bilinear")
    torch.cuda.synchronize()
    srv = gf.Server(slots=2)
    producer = torch.cuda.Stream()
    I = torch.zeros_like(src_I)
    p = torch.zeros_like(src_p)
    q = torch.full((1, C, H, W), float("nan"), device="cuda")
    with torch.cuda.stream(producer):
        torch.cuda._sleep(int(0.05 * 2.0e9))  # about 50 ms of GPU time before the inputs are written
        I.copy_(src_I)
        p.copy_(src_p)
        t = srv.submit(I, p, q, 8, 1e-2, 4, "bilinear")  # records its ready event on the producing stream
    res = srv.poll(t)
    srv.close()
    assert res["status"] == gf.GF_OK
    assert torch.equal(q, ref.view_as(q))


def test_request_whose_wait_runs_out_fails_alone(gf):
    """A request made to give up a bounded wait (gf_opts.test_wait_fault) is reported GF_EWAIT; the requests
    around it complete normally, and a request after it on the same slot is green."""
    I, p = _make(512, 1024, 3, torch.float32, 13)
    ref = gf.fast_guided_filter(I, p, 16, 1e-3, 4, "bilinear", fused=-1)
    torch.cuda.synchronize()
    gf.kernel_faults(clear=True)
    srv = gf.Server(slots=1)
    qs = [torch.full((1, 3, 512, 1024), -1.0, device="cuda") for _ in range(4)]
    tickets = [srv.submit(I, p, q, 16, 1e-3, 4, "bilinear", fused=-1, test_wait_fault=(k == 1))
               for k, q in enumerate(qs)]
    statuses = [srv.poll(t)["status"] for t in tickets]
    srv.close()
    assert statuses == [gf.GF_OK, gf.GF_EWAIT, gf.GF_OK, gf.GF_OK]
    for k in (0, 2, 3):
        assert torch.equal(qs[k], ref.view_as(qs[k]))
    assert gf.kernel_faults(clear=True) & 1
