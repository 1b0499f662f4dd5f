"""Synthetic scenes shaped like the paper's mega-pixel workloads.

The paper's own images (its figures) are not available, so seeded synthetic scenes stand in for them:
a smooth gradient, axis-aligned rectangles of uniform intensity (sharp edges for the edge-preserving
filter to keep), and Gaussian noise (texture for it to smooth), clipped to [0, 1] -- the value range on
which the paper's eps values (squared standard deviations) are quoted.

Recipe of ``make_scene(H, W, seed)``:
  1. I(y, x) = 0.5 * (x / (W - 1) + y / (H - 1))            (linear gradient; 0 on a 1-px axis)
  2. paint 20 rectangles over it, in order: intensity ~ U[0, 1], width ~ U[0.05, 0.5] * W,
     height ~ U[0.05, 0.5] * H, top-left corner uniform over the image, clipped to the image
  3. add N(0, 0.05^2) noise and clip to [0, 1]
All random draws come from ``numpy.random.default_rng(seed)`` (PCG64) in the order above, in float64;
the result is returned as float32.
"""
import numpy as np


def make_scene(H, W, seed=0, n_rects=20, noise_sigma=0.05):
    rng = np.random.default_rng(seed)
    ys = np.arange(H, dtype=np.float64)[:, None] / max(H - 1, 1)
    xs = np.arange(W, dtype=np.float64)[None, :] / max(W - 1, 1)
    img = 0.5 * (xs + ys)
    for _ in range(n_rects):
        val = rng.uniform(0.0, 1.0)
        rw = max(1, int(round(rng.uniform(0.05, 0.5) * W)))
        rh = max(1, int(round(rng.uniform(0.05, 0.5) * H)))
        x0 = int(rng.integers(0, W))
        y0 = int(rng.integers(0, H))
        img[y0:y0 + rh, x0:x0 + rw] = val
    img = img + rng.normal(0.0, noise_sigma, size=(H, W))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def make_color_scene(H, W, seed=0, n_rects=20, noise_sigma=0.05):
    """3 x H x W colour stand-in for the paper's application images: the recipe of ``make_scene`` with a
    colour per rectangle.  Draws, in order: per rectangle its colour (3 x U[0, 1]), width, height and
    top-left corner as in ``make_scene``; then N(0, noise_sigma^2) noise for the 3 planes."""
    rng = np.random.default_rng(seed)
    ys = np.arange(H, dtype=np.float64)[:, None] / max(H - 1, 1)
    xs = np.arange(W, dtype=np.float64)[None, :] / max(W - 1, 1)
    img = np.repeat((0.5 * (xs + ys))[None], 3, axis=0)
    for _ in range(n_rects):
        col = rng.uniform(0.0, 1.0, size=3)
        rw = max(1, int(round(rng.uniform(0.05, 0.5) * W)))
        rh = max(1, int(round(rng.uniform(0.05, 0.5) * H)))
        x0 = int(rng.integers(0, W))
        y0 = int(rng.integers(0, H))
        img[:, y0:y0 + rh, x0:x0 + rw] = col[:, None, None]
    img = img + rng.normal(0.0, noise_sigma, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def feather_mask(H, W, seed=4, n_shapes=3, block=16):
    """Coarse binary mask (float32 0 / 1), the input of guided feathering (the paper's Fig. 4): the union
    of ``n_shapes`` ellipses (centre uniform over the middle half of the image, semi-axes U[0.1, 0.3] x
    (W, H)), then made blocky by taking the value at the centre of each ``block`` x ``block`` cell -- a
    rough mask whose edges the guide is meant to refine."""
    rng = np.random.default_rng(seed)
    ys = np.arange(H, dtype=np.float64)[:, None]
    xs = np.arange(W, dtype=np.float64)[None, :]
    yc = (np.floor(ys / block) * block + block / 2.0).clip(0, H - 1)
    xc = (np.floor(xs / block) * block + block / 2.0).clip(0, W - 1)
    m = np.zeros((H, W), bool)
    for _ in range(n_shapes):
        cx, cy = rng.uniform(0.25, 0.75) * W, rng.uniform(0.25, 0.75) * H
        ax, ay = rng.uniform(0.1, 0.3) * W, rng.uniform(0.1, 0.3) * H
        m |= ((xc - cx) / ax) ** 2 + ((yc - cy) / ay) ** 2 <= 1.0
    return m.astype(np.float32)


def rgb_noisy_input(I, seed=1, channels=3, sigma=0.1):
    """p = I replicated per channel + independent N(0, sigma^2) noise, clipped to [0, 1] (float32)."""
    rng = np.random.default_rng(seed)
    I64 = np.asarray(I, np.float64)
    out = np.empty((channels,) + I64.shape, np.float32)
    for c in range(channels):
        out[c] = np.clip(I64 + rng.normal(0.0, sigma, size=I64.shape), 0.0, 1.0)
    return out


def quantize_u8(x):
    """Stored uint8 value: clamp(round_half_even(255 x), 0, 255)."""
    return np.clip(np.rint(np.asarray(x, np.float64) * 255.0), 0, 255).astype(np.uint8)


def to_f16_values(x):
    """Stored FP16 value of float32 data (round to nearest even)."""
    return np.asarray(x, np.float32).astype(np.float16)


def block_mean_downsample(x, s):
    """Mean of each s x s block (input recipe of the trainable-layer workload: its low-res p is the
    4x block-averaged guide plus noise).  Requires H and W divisible by s."""
    x = np.asarray(x, np.float64)
    *lead, H, W = x.shape
    if H % s or W % s:
        raise ValueError("block_mean_downsample needs sizes divisible by s")
    return x.reshape(*lead, H // s, s, W // s, s).mean(axis=(-3, -1))


def trainable_layer_batch(batch=16, channels=3, size=1024, s=4, seed0=3, noise_sigma=0.1):
    """Guide I (batch x channels x size x size, float32) built from scenes (rng seed seed0 + batch index,
    channels drawn in order), and low-res p = block mean of I by s + N(0, noise_sigma^2) (float32)."""
    I = np.empty((batch, channels, size, size), np.float32)
    p = np.empty((batch, channels, size // s, size // s), np.float32)
    for b in range(batch):
        rng = np.random.default_rng(seed0 + b)
        for c in range(channels):
            I[b, c] = make_scene(size, size, seed=int(rng.integers(0, 2**31 - 1)))
        low = block_mean_downsample(I[b], s)
        p[b] = (low + rng.normal(0.0, noise_sigma, size=low.shape)).astype(np.float32)
    return I, p


def serving_stream(n_requests=512, seed=2, rate_per_s=100.0, mp_range=(0.3, 24.0),
                   aspects=((4, 3), (16, 9), (1, 1)), channels=(1, 3), eps_choices=(1e-4, 1e-2),
                   s_choices=(4, 8)):
    """Seeded Poisson request stream for the serving workload.

    Each request: arrival time (exponential gaps at ``rate_per_s``), size drawn uniformly in megapixels,
    aspect ratio a uniform over ``aspects`` (W = round(sqrt(MP * 1e6 * a)), H = round(W / a)), channel
    count, r = round(0.004 * max(H, W)), eps and s uniform over their choices.  Returns a list of dicts.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        mp = rng.uniform(*mp_range)
        aw, ah = aspects[int(rng.integers(0, len(aspects)))]
        a = aw / ah
        W = max(1, int(round(np.sqrt(mp * 1e6 * a))))
        H = max(1, int(round(W / a)))
        C = int(channels[int(rng.integers(0, len(channels)))])
        r = int(round(0.004 * max(H, W)))
        eps = float(eps_choices[int(rng.integers(0, len(eps_choices)))])
        s = int(s_choices[int(rng.integers(0, len(s_choices)))])
        out.append(dict(id=k, arrival_s=t, H=H, W=W, C=C, r=r, eps=eps, s=s, scene_seed=1000 + k))
    return out
