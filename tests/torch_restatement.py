"""Float64 restatement of Algorithm 2 from PyTorch library routines, used only to pin the oracle.

Each step of the fast guided filter is delegated to an independent library routine whose behaviour is
documented, instead of re-typing the oracle's loops:
  box mean with border-normalised windows -> ``avg_pool2d(kernel 2r+1, stride 1, padding r,
                                              count_include_pad=False)``
  nearest subsample                       -> ``interpolate(mode="nearest-exact")``
  bilinear subsample / upsample           -> ``interpolate(mode="bilinear", align_corners=False,
                                              antialias=False)``
  box subsample                           -> ``avg_pool2d(kernel s, stride s, ceil_mode=True)``
The interpolate-based steps match the oracle's coordinate convention only when s divides H and W, so
the tests call this module on divisible sizes.  Being plain autograd-able torch code, it also provides a
float64 reference gradient for the hand-written backward pass.
"""
import torch
import torch.nn.functional as F


def box_mean(x, r):
    """x: (..., h, w) float64 -> window means over clipped windows of radius r."""
    shp = x.shape
    y = F.avg_pool2d(x.reshape(-1, 1, shp[-2], shp[-1]), kernel_size=2 * r + 1, stride=1, padding=r,
                     count_include_pad=False)
    return y.reshape(shp)


def subsample(x, s, mode):
    shp = x.shape
    H, W = shp[-2], shp[-1]
    h, w = -(-H // s), -(-W // s)
    x4 = x.reshape(-1, 1, H, W)
    if s == 1:
        y = x4
    elif mode == 0:
        y = F.interpolate(x4, size=(h, w), mode="nearest-exact")
    elif mode == 1:
        y = F.interpolate(x4, size=(h, w), mode="bilinear", align_corners=False, antialias=False)
    elif mode == 3:  # antialiased bilinear (divisible sizes: torch's scale is then exactly s)
        y = F.interpolate(x4, size=(h, w), mode="bilinear", align_corners=False, antialias=True)
    else:
        y = F.avg_pool2d(x4, kernel_size=s, stride=s, ceil_mode=True)
    return y.reshape(*shp[:-2], h, w)


def upsample(x, s, H, W):
    shp = x.shape
    if s == 1:
        return x
    y = F.interpolate(x.reshape(-1, 1, shp[-2], shp[-1]), size=(H, W), mode="bilinear", align_corners=False,
                      antialias=False)
    return y.reshape(*shp[:-2], H, W)


def fast_guided_filter(I, p, r_low, eps, s, mode, p_lowres=False):
    """I: (N, CI, H, W), p: (N, C, H, W) or (N, C, h, w); CI is 1 or C.  Returns q: (N, C, H, W)."""
    N, CI, H, W = I.shape
    C = p.shape[1]
    Ig = I.expand(N, C, H, W) if CI == 1 else I
    Il = subsample(Ig, s, mode)
    pl = p if p_lowres else subsample(p, s, mode)
    mean_I = box_mean(Il, r_low)
    mean_p = box_mean(pl, r_low)
    corr_I = box_mean(Il * Il, r_low)
    corr_Ip = box_mean(Il * pl, r_low)
    var_I = corr_I - mean_I * mean_I
    cov_Ip = corr_Ip - mean_I * mean_p
    a = cov_Ip / (var_I + eps)
    b = mean_p - a * mean_I
    mean_a = upsample(box_mean(a, r_low), s, H, W)
    mean_b = upsample(box_mean(b, r_low), s, H, W)
    return mean_a * Ig + mean_b


def color_guided_filter(I, p, r_low, eps, s, mode, p_lowres=False):
    """Colour-guided form: I (N, 3, H, W), p (N, C, H, W) or (N, C, h, w).  The 3 x 3 systems are solved
    with ``torch.linalg.solve``.  Returns q: (N, C, H, W)."""
    N, _, H, W = I.shape
    Il = subsample(I, s, mode)
    pl = p if p_lowres else subsample(p, s, mode)
    h, w = Il.shape[-2:]
    mean_I = box_mean(Il, r_low)                                             # (N, 3, h, w)
    sigma = box_mean(Il[:, :, None] * Il[:, None], r_low) - mean_I[:, :, None] * mean_I[:, None]
    mean_p = box_mean(pl, r_low)                                             # (N, C, h, w)
    cov = box_mean(Il[:, None] * pl[:, :, None], r_low) - mean_I[:, None] * mean_p[:, :, None]
    M = sigma.permute(0, 3, 4, 1, 2)[:, None] + eps * torch.eye(3, dtype=I.dtype)  # (N, 1, h, w, 3, 3)
    a = torch.linalg.solve(M.expand(N, pl.shape[1], h, w, 3, 3), cov.permute(0, 1, 3, 4, 2))
    a = a.permute(0, 1, 4, 2, 3)                                             # (N, C, 3, h, w)
    b = mean_p - (a * mean_I[:, None]).sum(2)
    mean_a = upsample(box_mean(a, r_low), s, H, W)
    mean_b = upsample(box_mean(b, r_low), s, H, W)
    return (mean_a * I[:, None]).sum(2) + mean_b
