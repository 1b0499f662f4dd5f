"""Trainable fast guided filter layer: a torch.autograd.Function over gf_filter / gf_filter_backward.

Forward and backward both run in libgf.so's CUDA kernels; this module only routes tensors.  The guide I,
the input p and eps all receive gradients (eps through a 0-dim tensor, so it can be a learnable parameter).
When a gradient is needed the forward keeps its low-res planes in the backward's workspace
(gf_opts.saved_forward), so the backward does not recompute them.
"""
from fractions import Fraction

import torch

from . import binding


class FastGuidedFilterFn(torch.autograd.Function):
    """q = FGF(I, p; r, eps, s).  Arguments: I, p (float32 CUDA, shapes as in ``fast_guided_filter``), eps (a
    0-dim float tensor or a Python float), r, s, mode, r_low, p_lowres."""

    @staticmethod
    def forward(ctx, I, p, eps, r, s=4, mode="bilinear", r_low=None, p_lowres=False):
        eps_val = float(eps.item()) if torch.is_tensor(eps) else float(eps)
        ws = None
        mode_id = binding.MODES[mode] if isinstance(mode, str) else int(mode)
        backward_ok = (I.dtype == torch.float32 and mode_id != binding.GF_SUB_BILINEAR_AA
                       and Fraction(s).denominator == 1)
        if any(ctx.needs_input_grad[:3]) and backward_ok:
            # the forward keeps its low-res planes in the backward's workspace, so the backward does not
            # recompute them
            I4 = I if I.dim() == 4 else I.reshape((1,) * (4 - I.dim()) + tuple(I.shape))
            p4 = p if p.dim() == 4 else p.reshape((1,) * (4 - p.dim()) + tuple(p.shape))
            nbytes = binding.backward_workspace_size(I4.shape[-2], I4.shape[-1], p4.shape[1], s, batch=I4.shape[0],
                                                     guide_channels=I4.shape[1], r_low=r_low, p_lowres=p_lowres)
            ws = torch.empty(nbytes, dtype=torch.uint8, device=I.device)
        q = binding.fast_guided_filter(I.detach(), p.detach(), r, eps_val, s, mode, r_low=r_low, p_lowres=p_lowres,
                                       workspace=ws, saved_forward=ws is not None)
        ctx.save_for_backward(I, p)
        ctx.ws = ws
        ctx.args = (r, eps_val, s, mode, r_low, p_lowres, torch.is_tensor(eps))
        return q

    @staticmethod
    def backward(ctx, dq):
        I, p = ctx.saved_tensors
        r, eps_val, s, mode, r_low, p_lowres, eps_is_tensor = ctx.args
        need_eps = eps_is_tensor and ctx.needs_input_grad[2]
        dI, dp, deps = binding.fast_guided_filter_backward(I.detach(), p.detach(), dq.contiguous(), r, eps_val, s, mode,
                                                           r_low=r_low, p_lowres=p_lowres, need_eps=need_eps,
                                                           workspace=ctx.ws, saved_forward=ctx.ws is not None)
        ctx.ws = None
        return (dI if ctx.needs_input_grad[0] else None, dp if ctx.needs_input_grad[1] else None,
                deps if need_eps else None, None, None, None, None, None)


class FastGuidedFilter(torch.nn.Module):
    """Guided-filter layer q = FGF(I, p) with a fixed radius and ratio and an optionally learnable eps."""

    def __init__(self, r, eps, s=4, mode="bilinear", r_low=None, p_lowres=False, learn_eps=False):
        super().__init__()
        self.r, self.s, self.mode, self.r_low, self.p_lowres = r, s, mode, r_low, p_lowres
        t = torch.tensor(float(eps), dtype=torch.float32)
        if learn_eps:
            self.eps = torch.nn.Parameter(t)
        else:
            self.register_buffer("eps", t)

    def forward(self, I, p):
        return FastGuidedFilterFn.apply(I, p, self.eps, self.r, self.s, self.mode, self.r_low, self.p_lowres)
