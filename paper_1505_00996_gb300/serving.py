"""Python front end of the serving loop (gf_submit / gf_poll / gf_cancel).

``Server`` owns a context whose scheduler thread admits queued filter requests as stream slots and HBM
budget free up; their kernels overlap on the GPU.  It keeps every submitted tensor alive until the request's
outcome has been collected, since the library reads I and p and writes q asynchronously.  Each submission
records an event on the stream that produced I and p (the current stream unless given), and the request's
kernels wait for it, so inputs still being written when submit is called are complete when they are read.
"""
import ctypes

import torch

from . import binding

_DTYPES = {torch.float32: binding.GF_F32, torch.float16: binding.GF_F16, torch.uint8: binding.GF_U8}


class Server:
    def __init__(self, device=None, hbm_budget_bytes=0, slots=4, queue_limit=0, graphs=False, tile_queue=True):
        """``graphs``: replay each request's launches through its bucket's CUDA graph (gf_serve_graphs).
        ``tile_queue``: run neighbouring single-kernel requests as one tile-queue launch (gf_serve_tile_queue)."""
        self.ctx = binding.Context(device, hbm_budget_bytes)
        self.lib = binding.load_library()
        binding.check(self.lib.gf_serve_config(self.ctx.handle, int(slots), int(queue_limit)))
        binding.check(self.lib.gf_serve_graphs(self.ctx.handle, int(bool(graphs))))
        binding.check(self.lib.gf_serve_tile_queue(self.ctx.handle, int(bool(tile_queue))))
        self._alive = {}

    def clock(self):
        return self.lib.gf_clock()

    def submit(self, I, p, q, r, eps, s=4, mode="bilinear", *, r_low=None, p_lowres=False, fused=0, stream=None,
               test_wait_fault=False):
        """Queue q = FGF(I, p).  I: (H, W) or (CI, H, W) or (N, CI, H, W) CUDA tensor; p likewise with C
        channels; q preallocated with the output shape and dtype.  ``stream``: the stream whose queued work
        writes I and p (default: the current stream).  ``test_wait_fault``: the timeout-path test hook of
        gf_opts.test_wait_fault.  Returns the ticket."""
        I4, _ = binding._nchw(I, "I")
        p4, _ = binding._nchw(p, "p")
        N, CI, H, W = I4.shape
        C = p4.shape[1]
        if not (I4.is_contiguous() and p4.is_contiguous() and q.is_contiguous()):
            raise ValueError("I, p and q must be contiguous")
        req = binding.GFRequest()
        self.lib.gf_opts_init(ctypes.byref(req.opts))
        req.I, req.p, req.q = I4.data_ptr(), p4.data_ptr(), q.data_ptr()
        req.H, req.W, req.C, req.r, req.eps = H, W, C, int(r), float(eps)
        req.s = binding._ratio(req.opts, s)  # a non-integer ratio travels in the options
        req.mode = binding.MODES[mode] if isinstance(mode, str) else int(mode)
        req.opts.batch = N
        req.opts.guide_channels = CI
        req.opts.r_low = -1 if r_low is None else int(r_low)
        req.opts.p_lowres = int(bool(p_lowres))
        req.opts.dtype_in = _DTYPES[I.dtype]
        req.opts.dtype_out = _DTYPES[q.dtype]
        req.opts.fused = int(fused)
        req.opts.test_wait_fault = int(bool(test_wait_fault))
        ready = torch.cuda.Event()
        ready.record(stream if stream is not None else torch.cuda.current_stream(I.device))
        req.ready_event = ready.cuda_event  # captured by gf_submit; the event may go once it returns
        ticket = ctypes.c_uint64()
        binding.check(self.lib.gf_submit(self.ctx.handle, ctypes.byref(req), ctypes.byref(ticket)))
        self._alive[ticket.value] = (I, p, q)
        return ticket.value

    def poll(self, ticket, timeout_s=None):
        """Outcome of a request: a dict with status and timestamps once it is terminal, or None if it is still
        pending (timeout_s = 0) / did not finish within timeout_s seconds.  timeout_s=None waits."""
        res = binding.GFResult()
        t_us = -1 if timeout_s is None else int(timeout_s * 1e6)
        st = self.lib.gf_poll(self.ctx.handle, ctypes.c_uint64(ticket), t_us, ctypes.byref(res))
        if st in (binding.GF_PENDING, binding.GF_ETIMEOUT):
            return None
        if st == binding.GF_ENOTFOUND:
            binding.check(st)
        self._alive.pop(ticket, None)
        return {"status": st, "ticket": res.ticket, "t_submit": res.t_submit, "t_admit": res.t_admit,
                "t_done": res.t_done, "scratch_bytes": res.scratch_bytes}

    def poll_status(self, ticket, timeout_us):
        """Raw gf_poll status (no result consumed unless terminal)."""
        res = binding.GFResult()
        st = self.lib.gf_poll(self.ctx.handle, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(res))
        if st not in (binding.GF_PENDING, binding.GF_ETIMEOUT):
            self._alive.pop(ticket, None)
        return st

    def cancel(self, ticket):
        return self.lib.gf_cancel(self.ctx.handle, ctypes.c_uint64(ticket))

    def pause(self, paused=True):
        binding.check(self.lib.gf_serve_pause(self.ctx.handle, int(bool(paused))))

    def stats(self):
        st = binding.GFServeStats()
        binding.check(self.lib.gf_serve_stats_get(self.ctx.handle, ctypes.byref(st)))
        return {"queued": st.queued, "running": st.running, "slots": st.slots, "budget_bytes": st.budget_bytes,
                "scratch_in_use": st.scratch_in_use, "launches": st.launches, "graph_launches": st.graph_launches,
                "queue_launches": st.queue_launches, "queue_requests": st.queue_requests,
                "launch_seconds": st.launch_seconds}

    def close(self):
        self.ctx.close()
        self._alive.clear()
