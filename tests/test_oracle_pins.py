"""Pins for the FP64 oracle: checks against things other than the oracle itself.

Each test ties one part of the oracle to an independent fact: hand-derived examples, brute force,
a library routine, the least-squares problem the coefficients solve, closed forms, invariances, or
finite differences.  A plausible slip anywhere in the oracle (dropped term, wrong sign or index,
transposed operand, wrong border count, off-by-half coordinate) fails at least one of them.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import torch_restatement as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------------------------------------------------
# Hand-derived examples (Eq. 2-4, Algorithms 1-2)
# ---------------------------------------------------------------------------------------------------------

def _frac_array(rows):
    return np.array([[float(Fraction(v)) for v in row] for row in rows])


@pytest.mark.parametrize("ex", json.load(open(GOLDEN))["examples"], ids=lambda e: e["name"])
def test_hand_examples(ex):
    q, inter = oracle.fast_guided_filter(np.array(ex["I"]), np.array(ex["p"]), ex["r"], ex["eps"], ex["s"],
                                         ex["mode"], r_low=ex["r_low"], intermediates=True)
    np.testing.assert_allclose(q, _frac_array(ex["q"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(inter["a"], _frac_array(ex["a"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(inter["b"], _frac_array(ex["b"]), rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------------------------------------
# Box mean f_mean (R1)
# ---------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_box_mean_matches_bruteforce(seed):
    rng = _rng(seed)
    for _ in range(12):
        h, w = int(rng.integers(1, 18)), int(rng.integers(1, 18))
        r = int(rng.integers(0, 20))
        x = rng.standard_normal((h, w))
        np.testing.assert_allclose(oracle.box_mean(x, r), oracle.box_mean_bruteforce(x, r), rtol=1e-13,
                                   atol=1e-14)


@pytest.mark.parametrize("shape,r", [((7, 11), 2), ((16, 9), 4), ((5, 5), 7), ((1, 13), 3), ((23, 1), 1),
                                     ((12, 12), 0)])
def test_box_mean_matches_avg_pool(shape, r):
    x = _rng(7).standard_normal(shape)
    ref = tr.box_mean(torch.from_numpy(x), r).numpy()
    np.testing.assert_allclose(oracle.box_mean(x, r), ref, rtol=1e-13, atol=1e-14)


def test_box_counts_closed_form():
    # sum of ones over a clipped window = (rows in window) * (cols in window)
    h, w, r = 9, 14, 3
    got = oracle.box_sum(np.ones((h, w)), r)
    ny = np.array([min(h - 1, j + r) - max(0, j - r) + 1 for j in range(h)])
    nx = np.array([min(w - 1, i + r) - max(0, i - r) + 1 for i in range(w)])
    np.testing.assert_array_equal(got, np.outer(ny, nx).astype(np.float64))
    np.testing.assert_allclose(oracle.box_mean(np.full((h, w), 0.37), r), 0.37, rtol=0, atol=1e-15)


def test_box_sum_integer_exact():
    x = _rng(3).integers(0, 1021, size=(31, 40)).astype(np.float64)
    got = oracle.box_sum(x, 4)
    # brute force in exact integers
    xi = x.astype(np.int64)
    ref = np.zeros_like(xi)
    for j in range(31):
        for i in range(40):
            ref[j, i] = xi[max(0, j - 4):j + 5, max(0, i - 4):i + 5].sum()
    np.testing.assert_array_equal(got.astype(np.int64), ref)
    assert np.all(got == np.round(got))


# ---------------------------------------------------------------------------------------------------------
# Subsample / upsample conventions (R2-R5, R7)
# ---------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [oracle.SUB_NEAREST, oracle.SUB_BILINEAR, oracle.SUB_BOX, oracle.SUB_BILINEAR_AA])
@pytest.mark.parametrize("s", [2, 3, 4, 8])
def test_subsample_matches_torch_divisible(mode, s):
    H, W = 5 * s, 3 * s
    x = _rng(s + 10 * mode).standard_normal((H, W))
    ref = tr.subsample(torch.from_numpy(x), s, mode).numpy()
    np.testing.assert_allclose(oracle.subsample(x, s, mode), ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("H,W,s", [(10, 13, 4), (7, 9, 3), (17, 5, 8), (9, 9, 2)])
def test_box_subsample_ragged_matches_avg_pool(H, W, s):
    x = _rng(H * W).standard_normal((H, W))
    ref = tr.subsample(torch.from_numpy(x), s, oracle.SUB_BOX).numpy()
    np.testing.assert_allclose(oracle.subsample(x, s, oracle.SUB_BOX), ref, rtol=1e-14, atol=1e-14)


def test_subsample_ragged_conventions():
    # R2/R3/R5 at a ragged edge: H = 10, s = 4 -> h = 3; last nearest row floor(2.5 * 4) = 10 -> clamped 9
    x = np.arange(10 * 6, dtype=np.float64).reshape(10, 6)
    near = oracle.subsample(x, 4, oracle.SUB_NEAREST)
    assert near.shape == (3, 2)
    assert near[2, 1] == x[9, 5] and near[0, 0] == x[2, 2] and near[1, 1] == x[6, 5]
    bil = oracle.subsample(x, 4, oracle.SUB_BILINEAR)
    # row 0 samples y = 1.5 (mean of rows 1 and 2); row 2 samples y = 9.5 -> clamped to 9
    assert bil[0, 0] == pytest.approx(x[1:3, 1:3].mean())
    assert bil[2, 0] == pytest.approx(x[9, 1:3].mean())


# ---------------------------------------------------------------------------------------------------------
# Non-integer ratios (R13): s = sn / sd with the same coordinate maps, decided exactly
# ---------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [oracle.SUB_NEAREST, oracle.SUB_BILINEAR, oracle.SUB_BILINEAR_AA])
@pytest.mark.parametrize("s", [Fraction(5, 2), Fraction(3, 2), Fraction(7, 4)])
def test_rational_subsample_matches_torch_scale_factor(mode, s):
    # torch maps output pixel j to (j + 1/2) / scale_factor - 1/2 when the scale factor is given and not
    # recomputed; with a binary fraction s that coordinate is exact, and the output has floor(H / s) rows
    # (ceil here), so the common part is compared
    H, W = 23, 17
    x = _rng(int(s * 4) + mode).standard_normal((H, W))
    torch_mode = {oracle.SUB_NEAREST: "nearest-exact", oracle.SUB_BILINEAR: "bilinear",
                  oracle.SUB_BILINEAR_AA: "bilinear"}[mode]
    kw = {} if mode == oracle.SUB_NEAREST else {"align_corners": False, "antialias": mode == oracle.SUB_BILINEAR_AA}
    ref = torch.nn.functional.interpolate(torch.from_numpy(x)[None, None], scale_factor=float(1 / s), mode=torch_mode,
                                          recompute_scale_factor=False, **kw)[0, 0].numpy()
    y = oracle.subsample(x, s, mode)
    assert y.shape == (-(-H * s.denominator // s.numerator), -(-W * s.denominator // s.numerator))
    hh, ww = ref.shape
    if mode == oracle.SUB_BILINEAR_AA:  # torch renormalises the clipped taps too; compare the interior
        np.testing.assert_allclose(y[1:hh - 1, 1:ww - 1], ref[1:hh - 1, 1:ww - 1], rtol=1e-13, atol=1e-13)
    else:
        np.testing.assert_allclose(y[:hh, :ww], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("s", [Fraction(5, 2), Fraction(3, 2), Fraction(9, 4)])
def test_rational_upsample_matches_torch_scale_factor(s):
    h, w = 7, 6
    x = _rng(int(s * 8)).standard_normal((h, w))
    H, W = int(h * s) - 1, int(w * s)
    ref = torch.nn.functional.interpolate(torch.from_numpy(x)[None, None], scale_factor=float(s), mode="bilinear",
                                          align_corners=False, recompute_scale_factor=False)[0, 0].numpy()
    np.testing.assert_allclose(oracle.upsample(x, s, H, W), ref[:H, :W], rtol=1e-13, atol=1e-13)


def test_rational_ratio_hand_values():
    s = Fraction(4, 3)  # not a binary fraction: positions decided exactly
    x = np.arange(7 * 5, dtype=np.float64).reshape(7, 5)
    near = oracle.subsample(x, s, oracle.SUB_NEAREST)  # rows floor((2j + 1) 2 / 3) = 0, 2, 3, 4, 6, (7 -> 6)
    assert near.shape == (6, 4)
    np.testing.assert_array_equal(near[:, 0], x[[0, 2, 3, 4, 6, 6], 0])
    bil = oracle.subsample(x, s, oracle.SUB_BILINEAR)  # rows ((2j + 1) 4 - 3) / 6 = 1/6, 3/2, 17/6, ...
    assert bil[0, 0] == pytest.approx(x[0, 0] + (x[1, 0] - x[0, 0]) / 6 + (x[0, 1] - x[0, 0]) / 6, abs=1e-12)
    assert bil[2, 0] == pytest.approx((1 - 5 / 6) * x[2, 0] + 5 / 6 * x[3, 0] + (x[2, 1] - x[2, 0]) / 6, abs=1e-12)
    up = oracle.upsample(np.arange(4.0)[None, :].repeat(2, 0), s, 2, 5)  # columns ((2X + 1) 3 - 4) / 8
    np.testing.assert_allclose(up[0], [0.0, 5 / 8, 11 / 8, 17 / 8, 23 / 8], atol=1e-15)
    assert oracle.lowres_radius(16, Fraction(5, 2)) == 6 and oracle.lowres_radius(5, s) == 4
    assert oracle.lowres_shape(10, 7, Fraction(5, 2)) == (4, 3)
    with pytest.raises(ValueError):
        oracle.subsample(x, s, oracle.SUB_BOX)


def test_integer_ratio_given_as_fraction_is_the_integer_ratio():
    rng = _rng(61)
    I = rng.uniform(0, 1, (1, 1, 24, 20))
    p = rng.uniform(0, 1, (1, 2, 24, 20))
    np.testing.assert_array_equal(oracle.fast_guided_filter(I, p, 8, 1e-2, Fraction(8, 2), oracle.SUB_BILINEAR),
                                  oracle.fast_guided_filter(I, p, 8, 1e-2, 4, oracle.SUB_BILINEAR))


def test_antialiased_subsample_hand_weights():
    # R11 at s = 4 along y on an image constant along x: interior rows take the taps 4j-2 .. 4j+5 with
    # weights (1, 3, 5, 7, 7, 5, 3, 1) / 32; the top row loses taps -2, -1 and renormalises the rest,
    # (5, 7, 7, 5, 3, 1) / 28; the bottom row of a 13-row image keeps only its taps 10, 11, 12: (1, 3, 5) / 9.
    rows = np.array([2.0, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41])
    x = np.repeat(rows[:, None], 8, axis=1)
    y = oracle.subsample(x, 4, oracle.SUB_BILINEAR_AA)
    assert y.shape == (4, 2)
    assert y[1, 0] == pytest.approx(np.dot([1, 3, 5, 7, 7, 5, 3, 1], rows[2:10]) / 32, abs=1e-14)
    assert y[0, 0] == pytest.approx(np.dot([5, 7, 7, 5, 3, 1], rows[0:6]) / 28, abs=1e-14)
    assert y[3, 1] == pytest.approx(np.dot([1, 3, 5], rows[10:13]) / 9, abs=1e-14)
    # odd s: s = 3 interior taps 3j-1 .. 3j+3 with weights (1, 2, 3, 2, 1) / 9
    y3 = oracle.subsample(x[:12], 3, oracle.SUB_BILINEAR_AA)
    assert y3[2, 0] == pytest.approx(np.dot([1, 2, 3, 2, 1], rows[5:10]) / 9, abs=1e-14)


def test_antialiased_subsample_keeps_constants():
    x = np.full((11, 14), 0.3)
    for s in (2, 3, 4, 8):
        np.testing.assert_allclose(oracle.subsample(x, s, oracle.SUB_BILINEAR_AA), 0.3, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mode", [oracle.SUB_NEAREST, oracle.SUB_BILINEAR, oracle.SUB_BOX, oracle.SUB_BILINEAR_AA])
def test_s1_subsample_is_identity(mode):
    x = _rng(5).standard_normal((6, 9))
    np.testing.assert_array_equal(oracle.subsample(x, 1, mode), x)
    np.testing.assert_array_equal(oracle.upsample(x, 1, 6, 9), x)


@pytest.mark.parametrize("s", [2, 4, 8])
def test_upsample_matches_torch(s):
    h, w = 6, 5
    x = _rng(s).standard_normal((h, w))
    ref = tr.upsample(torch.from_numpy(x), s, h * s, w * s).numpy()
    np.testing.assert_allclose(oracle.upsample(x, s, h * s, w * s), ref, rtol=1e-14, atol=1e-14)


def test_upsample_dyadic_phases_s4():
    # R7 at s = 4: interior pixels sit at offsets -3/8, -1/8, 1/8, 3/8 of a low-res cell
    x = np.array([[0.0, 8.0, 16.0]])
    up = oracle.upsample(x, 4, 1, 12)
    np.testing.assert_array_equal(up[0, 4:8], [5.0, 7.0, 9.0, 11.0])
    np.testing.assert_array_equal(up[0, :2], [0.0, 0.0])  # clamped left edge
    np.testing.assert_array_equal(up[0, 10:], [16.0, 16.0])


def test_lowres_radius_rule():
    assert oracle.lowres_radius(16, 4) == 4 and oracle.lowres_radius(8, 4) == 2
    assert oracle.lowres_radius(16, 8) == 2 and oracle.lowres_radius(60, 4) == 15
    assert oracle.lowres_radius(6, 4) == 2  # 1.5 rounds half up
    assert oracle.lowres_radius(3, 8) == 1  # raised to 1
    assert oracle.lowres_radius(0, 4) == 0 and oracle.lowres_radius(7, 1) == 7


# ---------------------------------------------------------------------------------------------------------
# Coefficients: Eq. (2)-(3) are the minimiser of the windowed ridge regression
# ---------------------------------------------------------------------------------------------------------

def _ridge_coefficients(I, p, r, eps):
    """For every clipped window, minimise sum_i (a I_i + b - p_i)^2 + eps a^2 with a least-squares
    solver (the reconstruction error the paper's coefficients minimise)."""
    h, w = I.shape
    a = np.empty((h, w))
    b = np.empty((h, w))
    for j in range(h):
        for i in range(w):
            sl = (slice(max(0, j - r), j + r + 1), slice(max(0, i - r), i + r + 1))
            Iw, pw = I[sl].ravel(), p[sl].ravel()
            n = Iw.size
            A = np.concatenate([np.stack([Iw, np.ones(n)], 1), np.tile([[np.sqrt(eps), 0.0]], (n, 1))])
            rhs = np.concatenate([pw, np.zeros(n)])
            sol = np.linalg.lstsq(A, rhs, rcond=None)[0]
            a[j, i], b[j, i] = sol
    return a, b


@pytest.mark.parametrize("seed,r,eps", [(0, 1, 0.01), (1, 2, 0.1), (2, 3, 1e-3), (3, 6, 0.04)])
def test_coefficients_solve_ridge_regression(seed, r, eps):
    rng = _rng(seed)
    H, W = 9, 12
    I = rng.uniform(0, 1, (H, W))
    p = rng.uniform(0, 1, (H, W))
    q, inter = oracle.fast_guided_filter(I, p, r, eps, 1, intermediates=True)
    a_ref, b_ref = _ridge_coefficients(I, p, r, eps)
    np.testing.assert_allclose(inter["a"], a_ref, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(inter["b"], b_ref, rtol=1e-9, atol=1e-10)
    # Eq. (4): q_i is the average over the windows that contain i of a_k I_i + b_k
    q_ref = np.empty_like(I)
    for j in range(H):
        for i in range(W):
            ks = [(jj, ii) for jj in range(max(0, j - r), min(H, j + r + 1))
                  for ii in range(max(0, i - r), min(W, i + r + 1))]
            q_ref[j, i] = np.mean([a_ref[k] * I[j, i] + b_ref[k] for k in ks])
    np.testing.assert_allclose(q, q_ref, rtol=1e-9, atol=1e-10)


# ---------------------------------------------------------------------------------------------------------
# Whole filter
# ---------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed,H,W,r,eps", [(0, 20, 17, 3, 0.01), (1, 8, 31, 5, 1e-3), (2, 33, 6, 2, 0.2)])
def test_s1_equals_separately_coded_guided_filter(seed, H, W, r, eps):
    rng = _rng(seed)
    I = rng.uniform(0, 1, (H, W))
    p = rng.uniform(0, 1, (H, W))
    for mode in (oracle.SUB_NEAREST, oracle.SUB_BILINEAR, oracle.SUB_BOX):
        q_fgf = oracle.fast_guided_filter(I, p, r, eps, 1, mode)
        np.testing.assert_allclose(q_fgf, oracle.guided_filter(I, p, r, eps), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("s,mode,CI", [(2, 0, 1), (4, 1, 1), (4, 2, 3), (8, 1, 3), (3, 0, 3), (1, 1, 1), (4, 3, 1),
                                       (3, 3, 3), (Fraction(5, 2), 1, 1), (Fraction(3, 2), 0, 3),
                                       (Fraction(5, 2), 3, 1)])
def test_fgf_matches_torch_restatement(s, mode, CI):
    # sizes are multiples of sn, so the low-res grid is H sd / sn and torch's size-based scale equals s
    rng = _rng(int(s * 10) + mode)
    N, C, H, W = 2, 3, 6 * Fraction(s).numerator, 5 * Fraction(s).numerator
    I = rng.uniform(0, 1, (N, CI, H, W))
    p = rng.uniform(0, 1, (N, C, H, W))
    r_low = 2
    q = oracle.fast_guided_filter(I, p, 0, 0.02, s, mode, r_low=r_low)
    ref = tr.fast_guided_filter(torch.from_numpy(I), torch.from_numpy(p), r_low, 0.02, s, mode).numpy()
    np.testing.assert_allclose(q, ref, rtol=1e-11, atol=1e-12)


def test_fgf_lowres_p_matches_torch_restatement():
    rng = _rng(42)
    s, N, C, H, W = 4, 2, 3, 32, 24
    I = rng.uniform(0, 1, (N, C, H, W))
    p = rng.uniform(0, 1, (N, C, H // s, W // s))
    q = oracle.fast_guided_filter(I, p, 0, 1e-2, s, oracle.SUB_BOX, r_low=2, p_lowres=True)
    ref = tr.fast_guided_filter(torch.from_numpy(I), torch.from_numpy(p), 2, 1e-2, s, 2, p_lowres=True).numpy()
    np.testing.assert_allclose(q, ref, rtol=1e-11, atol=1e-12)


def test_brute_and_separable_box_backends_agree():
    rng = _rng(9)
    I = rng.uniform(0, 1, (1, 1, 19, 23))
    p = rng.uniform(0, 1, (1, 2, 19, 23))
    for s, mode in [(1, 1), (2, 0), (3, 1), (4, 2)]:
        a = oracle.fast_guided_filter(I, p, 5, 1e-2, s, mode)
        b = oracle.fast_guided_filter(I, p, 5, 1e-2, s, mode, brute=True)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-13)


def test_constant_p_gives_constant_q():
    rng = _rng(11)
    I = rng.uniform(0, 1, (30, 41))
    for s, mode in [(1, 1), (4, 1), (3, 0), (4, 2)]:
        q = oracle.fast_guided_filter(I, np.full((30, 41), 0.625), 8, 1e-3, s, mode)
        np.testing.assert_allclose(q, 0.625, rtol=0, atol=1e-13)


def test_constant_guide_gives_double_box_mean_of_p():
    # var = cov = 0 -> a = 0, b = mean_p, q = mean of mean_p; far from the border this is the plain
    # (2r'+1)^2 double box mean, which a 2-D convolution with a uniform kernel computes independently.
    rng = _rng(12)
    H = W = 40
    p = rng.uniform(0, 1, (H, W))
    # a power-of-two guide value keeps every window sum exact, so var and cov are exactly zero
    q, inter = oracle.fast_guided_filter(np.full((H, W), 0.5), p, 3, 1e-2, 1, intermediates=True)
    assert np.all(inter["a"] == 0.0)
    k = np.ones((7, 7)) / 49.0
    from scipy.signal import convolve2d
    dbl = convolve2d(convolve2d(p, k, mode="valid"), k, mode="valid")
    np.testing.assert_allclose(q[6:-6, 6:-6], dbl, rtol=1e-12, atol=1e-13)


def test_affine_p_closed_form():
    # p = alpha I + beta (s = 1): cov = alpha var, so a = alpha var / (var + eps) with var the windowed
    # variance (computed here two-pass, as the mean squared deviation), b = mean_p - a mean_I.
    rng = _rng(13)
    H, W, r, eps, alpha, beta = 14, 15, 2, 0.05, 0.7, 0.1
    I = rng.uniform(0, 1, (H, W))
    _, inter = oracle.fast_guided_filter(I, alpha * I + beta, r, eps, 1, intermediates=True)
    var = np.empty((H, W))
    mu = np.empty((H, W))
    for j in range(H):
        for i in range(W):
            win = I[max(0, j - r):j + r + 1, max(0, i - r):i + r + 1]
            mu[j, i] = win.mean()
            var[j, i] = ((win - win.mean()) ** 2).mean()
    a_ref = alpha * var / (var + eps)
    np.testing.assert_allclose(inter["a"], a_ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(inter["b"], alpha * mu + beta - a_ref * mu, rtol=1e-10, atol=1e-12)
    # eps -> 0: q -> p
    q0 = oracle.fast_guided_filter(I, alpha * I + beta, r, 1e-12, 1)
    np.testing.assert_allclose(q0, alpha * I + beta, rtol=0, atol=1e-8)


def test_invariances():
    rng = _rng(14)
    H, W, r, eps, s = 24, 28, 8, 1e-2, 4
    I = rng.uniform(0, 1, (H, W))
    p1 = rng.uniform(0, 1, (H, W))
    p2 = rng.uniform(0, 1, (H, W))
    f = lambda I_, p_, e=eps: oracle.fast_guided_filter(I_, p_, r, e, s, oracle.SUB_BILINEAR)
    # linear in p
    np.testing.assert_allclose(f(I, 2.0 * p1 - 3.0 * p2), 2.0 * f(I, p1) - 3.0 * f(I, p2), atol=1e-12)
    # shift of the guide
    np.testing.assert_allclose(f(I + 0.25, p1), f(I, p1), atol=1e-12)
    # scaling the guide by k and eps by k^2
    np.testing.assert_allclose(f(3.0 * I, p1, 9.0 * eps), f(I, p1), atol=1e-12)


def test_depthwise_guide_channels():
    rng = _rng(15)
    I = rng.uniform(0, 1, (1, 3, 16, 20))
    p = rng.uniform(0, 1, (1, 3, 16, 20))
    q = oracle.fast_guided_filter(I, p, 4, 1e-2, 2, oracle.SUB_BILINEAR)
    for c in range(3):
        qc = oracle.fast_guided_filter(I[0, c], p[0, c], 4, 1e-2, 2, oracle.SUB_BILINEAR)
        np.testing.assert_array_equal(q[0, c], qc)


# ---------------------------------------------------------------------------------------------------------
# Colour guide (R12): the guided filter's colour form inside Algorithm 2
# ---------------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("s,mode", [(1, 1), (2, 0), (4, 1), (4, 2), (3, 3)])
def test_color_guide_of_replicated_gray_equals_gray_guide_with_eps_over_3(s, mode):
    # I_r = I_g = I_b = G makes Sigma = var 11^T and cov_Ip = cov 1, so (Sigma + eps U)^-1 cov_Ip =
    # cov / (3 var + eps) 1 and a^T I = cov / (var + eps / 3) G: the gray filter with eps / 3
    rng = _rng(20 + s)
    G = rng.uniform(0, 1, (2, 1, 6 * s, 5 * s))
    p = rng.uniform(0, 1, (2, 3, 6 * s, 5 * s))
    q_col = oracle.color_guided_filter(np.repeat(G, 3, axis=1), p, 0, 3e-2, s, mode, r_low=2)
    q_gray = oracle.fast_guided_filter(G, p, 0, 1e-2, s, mode, r_low=2)
    np.testing.assert_allclose(q_col, q_gray, rtol=0, atol=1e-12)


def _ridge_coefficients_color(I, p, r, eps):
    """For every clipped window, minimise sum_i (a^T I_i + b - p_i)^2 + n eps |a|^2 (n = window size) with a
    least-squares solver."""
    _, h, w = I.shape
    a = np.empty((3, h, w))
    b = np.empty((h, w))
    for j in range(h):
        for i in range(w):
            sl = (slice(None), slice(max(0, j - r), j + r + 1), slice(max(0, i - r), i + r + 1))
            Iw = I[sl].reshape(3, -1).T
            pw = p[sl[1:]].ravel()
            n = pw.size
            A = np.concatenate([np.concatenate([Iw, np.ones((n, 1))], 1),
                                np.concatenate([np.sqrt(n * eps) * np.eye(3), np.zeros((3, 1))], 1)])
            sol = np.linalg.lstsq(A, np.concatenate([pw, np.zeros(3)]), rcond=None)[0]
            a[:, j, i], b[j, i] = sol[:3], sol[3]
    return a, b


@pytest.mark.parametrize("seed,r,eps", [(0, 1, 0.01), (1, 2, 1e-3), (2, 4, 0.1)])
def test_color_coefficients_solve_ridge_regression(seed, r, eps):
    rng = _rng(30 + seed)
    I = rng.uniform(0, 1, (3, 9, 11))
    p = rng.uniform(0, 1, (9, 11))
    _, inter = oracle.color_guided_filter(I, p[None], r, eps, 1, oracle.SUB_BILINEAR, intermediates=True)
    a_ref, b_ref = _ridge_coefficients_color(I, p, r, eps)
    np.testing.assert_allclose(inter["a"][0, 0], a_ref, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(inter["b"][0, 0], b_ref, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("s,mode", [(1, 1), (2, 1), (4, 0), (4, 2), (4, 3), (8, 1)])
def test_color_guide_matches_torch_restatement(s, mode):
    rng = _rng(40 + s + mode)
    N, C, H, W = 2, 2, 5 * s, 7 * s
    I = rng.uniform(0, 1, (N, 3, H, W))
    p = rng.uniform(0, 1, (N, C, H, W))
    q = oracle.color_guided_filter(I, p, 0, 1e-2, s, mode, r_low=2)
    ref = tr.color_guided_filter(torch.from_numpy(I), torch.from_numpy(p), 2, 1e-2, s, mode).numpy()
    np.testing.assert_allclose(q, ref, rtol=1e-10, atol=1e-11)


def test_color_guide_lowres_p_matches_torch_restatement():
    rng = _rng(47)
    s, N, C, H, W = 4, 2, 3, 28, 20
    I = rng.uniform(0, 1, (N, 3, H, W))
    p = rng.uniform(0, 1, (N, C, H // s, W // s))
    q = oracle.color_guided_filter(I, p, 0, 1e-2, s, oracle.SUB_BOX, r_low=2, p_lowres=True)
    ref = tr.color_guided_filter(torch.from_numpy(I), torch.from_numpy(p), 2, 1e-2, s, 2, p_lowres=True).numpy()
    np.testing.assert_allclose(q, ref, rtol=1e-10, atol=1e-11)


def test_color_guide_closed_forms_and_invariances():
    rng = _rng(50)
    I = rng.uniform(0, 1, (1, 3, 24, 32))
    f = lambda I_, p_, e=1e-2: oracle.color_guided_filter(I_, p_, 8, e, 4, oracle.SUB_BILINEAR)
    # constant p gives back the constant exactly in exact arithmetic (a = 0, b = c)
    np.testing.assert_allclose(f(I, np.full((1, 1, 24, 32), 0.625)), 0.625, rtol=0, atol=1e-13)
    # p = alpha^T I + beta with eps = 0: a = alpha, b = beta everywhere, so q = p
    alpha, beta = np.array([0.5, -0.25, 0.75]), 0.125
    p_lin = (alpha[None, :, None, None] * I).sum(1, keepdims=True) + beta
    np.testing.assert_allclose(oracle.color_guided_filter(I, p_lin, 4, 0.0, 1, oracle.SUB_BILINEAR), p_lin,
                               rtol=0, atol=1e-9)
    # linear in p; a shift of every guide channel changes nothing
    p1, p2 = rng.uniform(0, 1, (2, 1, 2, 24, 32))
    np.testing.assert_allclose(f(I, 2.0 * p1 - 3.0 * p2), 2.0 * f(I, p1) - 3.0 * f(I, p2), atol=1e-12)
    np.testing.assert_allclose(f(I + np.array([0.1, -0.2, 0.3])[None, :, None, None], p1), f(I, p1), atol=1e-12)


# ---------------------------------------------------------------------------------------------------------
# Detail enhancement (the application of Fig. 2: base layer q plus k times the detail layer I - q)
# ---------------------------------------------------------------------------------------------------------

def test_detail_enhance_special_gains():
    rng = _rng(16)
    I = rng.uniform(0, 1, (1, 3, 20, 24))
    q = rng.uniform(0, 1, (1, 3, 20, 24))
    out = lambda k, I_=I: oracle.detail_enhance(I_, q, k)
    np.testing.assert_array_equal(out(0.0), q)               # no detail: the base layer
    np.testing.assert_allclose(out(1.0), I, atol=1e-15)      # all of the detail: the guide itself
    np.testing.assert_allclose(out(5.0) - q, 5.0 * (out(1.0) - q), atol=1e-13)  # the detail scales with k
    # a gray guide serves every channel
    Ig = I[:, :1]
    np.testing.assert_array_equal(out(2.0, Ig)[0, 2], oracle.detail_enhance(Ig[0, 0], q[0, 2], 2.0))


def test_detail_enhance_of_constant_image_is_the_image():
    # a constant image filtered with itself as guide is returned unchanged (a = 0, b = c), so its
    # enhanced version at any gain is the image again
    I = np.full((24, 32), 0.375)
    q = oracle.fast_guided_filter(I, I, 8, 1e-2, 4, oracle.SUB_BILINEAR)
    np.testing.assert_array_equal(oracle.detail_enhance(I, q, 5.0), I)


# ---------------------------------------------------------------------------------------------------------
# Backward pass
# ---------------------------------------------------------------------------------------------------------

def _loss(I, p, Wt, r_low, eps, s, mode, p_lowres):
    q = oracle.fast_guided_filter(I, p, 0, eps, s, mode, r_low=r_low, p_lowres=p_lowres)
    return float(np.sum(q * Wt))


@pytest.mark.parametrize("s,mode,CI,p_lowres", [(1, 1, 1, False), (2, 1, 1, False), (2, 0, 3, False),
                                                (3, 2, 2, False), (2, 2, 2, True), (3, 1, 1, False)])
def test_backward_central_differences(s, mode, CI, p_lowres):
    # (odd s with bilinear subsampling puts every sample on a pixel, weights 1 and 0; even s gives 1/2 and
    # 1/2, where a swapped weight of the transposed subsample would go unseen)
    rng = _rng(20 + s + mode)
    N, C, H, W, r_low, eps, hstep = 1, 2, 7, 6, 1, 0.05, 1e-3
    CI = 1 if CI == 1 else C
    I = rng.uniform(0, 1, (N, CI, H, W))
    hl, wl = oracle.lowres_shape(H, W, s)
    p = rng.uniform(0, 1, (N, C, hl, wl) if p_lowres else (N, C, H, W))
    Wt = rng.uniform(-1, 1, (N, C, H, W))
    dI, dp, deps = oracle.fast_guided_filter_backward(I, p, Wt, 0, eps, s, mode, r_low=r_low, p_lowres=p_lowres)
    for arr, grad in ((I, dI), (p, dp)):
        fd = np.empty_like(arr)
        it = np.nditer(arr, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = arr[idx]
            arr[idx] = old + hstep
            lp = _loss(I, p, Wt, r_low, eps, s, mode, p_lowres)
            arr[idx] = old - hstep
            lm = _loss(I, p, Wt, r_low, eps, s, mode, p_lowres)
            arr[idx] = old
            fd[idx] = (lp - lm) / (2 * hstep)
        np.testing.assert_allclose(grad, fd, rtol=2e-5, atol=2e-6)
    # q is a rational function of eps with curvature on the scale of eps itself, so the central difference
    # is Richardson-extrapolated (error O(h^4)) instead of taken at one step
    cd = lambda hh: (_loss(I, p, Wt, r_low, eps + hh, s, mode, p_lowres) -
                     _loss(I, p, Wt, r_low, eps - hh, s, mode, p_lowres)) / (2 * hh)
    fd_eps = (4.0 * cd(hstep / 2) - cd(hstep)) / 3.0
    assert deps == pytest.approx(fd_eps, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("s,mode,CI", [(1, 1, 1), (4, 1, 1), (4, 2, 3), (2, 0, 3)])
def test_backward_matches_torch_autograd(s, mode, CI):
    rng = _rng(30 + s)
    N, C, H, W, r_low, eps = 2, 3, 4 * s, 3 * s, 2, 1e-2
    I = rng.uniform(0, 1, (N, CI, H, W))
    p = rng.uniform(0, 1, (N, C, H, W))
    Wt = rng.uniform(-1, 1, (N, C, H, W))
    dI, dp, deps = oracle.fast_guided_filter_backward(I, p, Wt, 0, eps, s, mode, r_low=r_low)
    tI = torch.tensor(I, requires_grad=True)
    tp = torch.tensor(p, requires_grad=True)
    te = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    (tr.fast_guided_filter(tI, tp, r_low, te, s, mode) * torch.from_numpy(Wt)).sum().backward()
    np.testing.assert_allclose(dI, tI.grad.numpy(), rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(dp, tp.grad.numpy(), rtol=1e-10, atol=1e-11)
    assert deps == pytest.approx(te.grad.item(), rel=1e-10, abs=1e-11)


def test_backward_lowres_p_batch_matches_torch_autograd():
    """The trainable-layer form: a batch of low-res p (box subsample of the guide, s = 4)."""
    rng = _rng(35)
    s, N, C, H, W, r_low, eps = 4, 2, 3, 16, 12, 2, 1e-2
    I = rng.uniform(0, 1, (N, C, H, W))
    p = rng.uniform(0, 1, (N, C, H // s, W // s))
    Wt = rng.uniform(-1, 1, (N, C, H, W))
    dI, dp, deps = oracle.fast_guided_filter_backward(I, p, Wt, 0, eps, s, oracle.SUB_BOX, r_low=r_low, p_lowres=True)
    tI = torch.tensor(I, requires_grad=True)
    tp = torch.tensor(p, requires_grad=True)
    te = torch.tensor(eps, dtype=torch.float64, requires_grad=True)
    (tr.fast_guided_filter(tI, tp, r_low, te, s, 2, p_lowres=True) * torch.from_numpy(Wt)).sum().backward()
    np.testing.assert_allclose(dI, tI.grad.numpy(), rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(dp, tp.grad.numpy(), rtol=1e-10, atol=1e-11)
    assert deps == pytest.approx(te.grad.item(), rel=1e-10, abs=1e-11)


def test_backward_brute_and_separable_agree():
    rng = _rng(33)
    I = rng.uniform(0, 1, (1, 1, 13, 11))
    p = rng.uniform(0, 1, (1, 2, 13, 11))
    Wt = rng.uniform(-1, 1, (1, 2, 13, 11))
    a = oracle.fast_guided_filter_backward(I, p, Wt, 0, 1e-2, 2, 1, r_low=3)
    b = oracle.fast_guided_filter_backward(I, p, Wt, 0, 1e-2, 2, 1, r_low=3, brute=True)
    for x, y in zip(a[:2], b[:2]):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-13)
    assert a[2] == pytest.approx(b[2], rel=1e-12)


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.fast_guided_filter(np.ones((2, 3, 4, 4)), np.ones((2, 2, 4, 4)), 1, 0.1, 1)  # CI not 1 or C
    with pytest.raises(ValueError):
        oracle.fast_guided_filter(np.ones((4, 4)), np.ones((4, 4)), 1, -0.1, 1)
