"""Mutation check of the oracle's pins (CPU).

Each case plants one plausible mistake in a copy of ``oracle/gf_oracle.c`` -- a wrong border count, a
half-pixel offset, a dropped or mis-signed term of Eq. 2-4, a skipped step of Algorithm 2, a wrong factor in
the adjoint, a mis-scaled regulariser in the colour solve -- builds the copy with the oracle's own compiler
flags, and runs a selection of the pins of ``test_oracle_pins.py`` on it.  At least one pin must fail for
every planted mistake, and every pin must pass on an unmodified copy built the same way, so the pins are
shown to catch these mistakes rather than assumed to.  The mistakes change arithmetic or clamped indices
only, never a loop bound or an allocation, so a planted build cannot read or write out of bounds.  The
oracle's own build is not touched: the copies go to ``oracle/_build/mutants`` and are loaded through
``oracle.use_library`` for the duration of one case.
"""
import json
import os
import zlib
from fractions import Fraction

import pytest

import oracle
import test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gf_oracle.c")
OUT = os.path.join(ROOT, "oracle", "_build", "mutants")
EXAMPLES = json.load(open(pins.GOLDEN))["examples"]


def _each(fn, cases):
    return lambda: [fn(*c) for c in cases]


# The pins run on every build: (name, callable that raises when the pin does not hold).
PINS = [
    ("hand examples (Eq. 2-4)", lambda: [pins.test_hand_examples(ex) for ex in EXAMPLES]),
    ("box mean vs avg_pool2d", _each(pins.test_box_mean_matches_avg_pool, [((7, 11), 2), ((5, 5), 7), ((1, 13), 3)])),
    ("separable box mean vs brute-force windows", _each(pins.test_box_mean_matches_bruteforce, [(0,), (1,)])),
    ("brute-force and separable back ends agree",
     lambda: [pins.test_brute_and_separable_box_backends_agree(), pins.test_backward_brute_and_separable_agree()]),
    ("subsample vs torch interpolate / avg_pool2d",
     _each(pins.test_subsample_matches_torch_divisible, [(m, s) for m in range(4) for s in (2, 3, 4)])),
    ("ragged box subsample vs avg_pool2d", _each(pins.test_box_subsample_ragged_matches_avg_pool, [(10, 13, 4), (7, 9, 3)])),
    ("upsample vs torch interpolate", _each(pins.test_upsample_matches_torch, [(2,), (4,)])),
    ("r' rule", pins.test_lowres_radius_rule),
    ("Eq. 2-3 solve the ridge regression", _each(pins.test_coefficients_solve_ridge_regression, [(1, 2, 0.1)])),
    ("s = 1 equals the separately coded Algorithm 1",
     _each(pins.test_s1_equals_separately_coded_guided_filter, [(0, 20, 17, 3, 0.01)])),
    ("whole filter vs the float64 torch restatement",
     _each(pins.test_fgf_matches_torch_restatement, [(2, 0, 1), (4, 1, 1), (4, 2, 3), (4, 3, 1)])),
    ("backward vs central differences",
     _each(pins.test_backward_central_differences,
           [(2, 1, 1, False), (3, 1, 1, False), (3, 2, 2, False), (2, 0, 3, False), (2, 2, 2, True)])),
    ("backward vs float64 autograd", _each(pins.test_backward_matches_torch_autograd, [(4, 1, 1), (2, 0, 3)])),
    ("backward of a low-res p batch vs float64 autograd", pins.test_backward_lowres_p_batch_matches_torch_autograd),
    ("colour: replicated gray guide equals gray guide with eps / 3",
     _each(pins.test_color_guide_of_replicated_gray_equals_gray_guide_with_eps_over_3, [(2, 0), (4, 1)])),
    ("colour vs the float64 torch restatement", _each(pins.test_color_guide_matches_torch_restatement, [(4, 1)])),
    ("low-res p vs the float64 torch restatement",
     lambda: [pins.test_fgf_lowres_p_matches_torch_restatement(), pins.test_color_guide_lowres_p_matches_torch_restatement()]),
    ("detail epilogue special gains", pins.test_detail_enhance_special_gains),
    ("non-integer ratios vs torch interpolate",
     lambda: ([pins.test_rational_subsample_matches_torch_scale_factor(m, s)
               for m in (0, 1, 3) for s in (Fraction(5, 2), Fraction(7, 4))] +
              [pins.test_rational_upsample_matches_torch_scale_factor(s) for s in (Fraction(5, 2), Fraction(9, 4))])),
    ("non-integer ratio hand values", pins.test_rational_ratio_hand_values),
]

# (name, text of gf_oracle.c, the same text with the mistake planted)
MUTATIONS = [
    ("unclipped window count (R1)",
     "    int ny = imin(h - 1, j + r) - imax(0, j - r) + 1;",
     "    int ny = 2 * r + 1;"),
    ("nearest subsample without the half-pixel offset (R2)",
     "int sy = iclamp((int)(((2LL * j + 1) * sn) / (2LL * sd)), 0, H - 1);",
     "int sy = iclamp((int)(((2LL * j) * sn) / (2LL * sd)), 0, H - 1);"),
    ("bilinear subsample off by half a pixel (R3)",
     "axis_taps_q((2LL * j + 1) * sn - sd, 2LL * sd, H, &y0, &y1, &fy);",
     "axis_taps_q((2LL * j + 1) * sn, 2LL * sd, H, &y0, &y1, &fy);"),
    ("box subsample dividing ragged blocks by s^2 (R4)",
     "v = acc / (double)((yb - ya) * (xb - xa));",
     "v = acc / (double)(sn * sn);"),
    ("antialiased subsample with a wider triangle (R11)",
     "long long num = 2LL * sn - (d < 0 ? -d : d);",
     "long long num = 3LL * sn - (d < 0 ? -d : d);"),
    ("upsample off by half a pixel (R7)",
     "axis_taps_q((2LL * X + 1) * sd - sn, 2LL * sn, w, &x0, &x1, &fx);",
     "axis_taps_q((2LL * X + 1) * sd, 2LL * sn, w, &x0, &x1, &fx);"),
    ("upsample reading the upper tap row twice (R7)",
     "            double bot = (1.0 - fx) * x[(size_t)y1 * w + x0] + fx * x[(size_t)y1 * w + x1];",
     "            double bot = (1.0 - fx) * x[(size_t)y0 * w + x0] + fx * x[(size_t)y0 * w + x1];"),
    ("r' truncated instead of rounded half up (R6)",
     "int rl = (int)((2LL * r * sd + sn) / (2LL * sn));",
     "int rl = (int)((2LL * r * sd) / (2LL * sn));"),
    ("variance without the squared mean (Alg. 2)",
     "double var_I = corr_I[k] - mean_I[k] * mean_I[k];",
     "double var_I = corr_I[k];"),
    ("covariance without the product of means (Alg. 2)",
     "double cov_Ip = corr_Ip[k] - mean_I[k] * mean_p[k];",
     "double cov_Ip = corr_Ip[k];"),
    ("eps squared in Eq. 2",
     "a[k] = cov_Ip / (var_I + eps);",
     "a[k] = cov_Ip / (var_I + eps * eps);"),
    ("wrong sign of b in Eq. 3",
     "b[k] = mean_p[k] - a[k] * mean_I[k];",
     "b[k] = mean_p[k] + a[k] * mean_I[k];"),
    ("second box mean of b skipped (Alg. 2)",
     "box_mean_mode(b, h, w, r_low, brute, mean_b);",
     "memcpy(mean_b, b, sizeof(double) * n);"),
    ("output terms swapped in Eq. 4",
     "qc[k] = up_a[k] * Ig[k] + up_b[k];",
     "qc[k] = up_b[k] * Ig[k] + up_a[k];"),
    ("Algorithm 1 variance without the squared mean",
     "double var = cI[k] - mI[k] * mI[k];",
     "double var = cI[k];"),
    ("adjoint: wrong sign of d var",
     "double dvar = -da_k * a[k] * inv;",
     "double dvar = da_k * a[k] * inv;"),
    ("adjoint: factor 2 of d mean_I dropped",
     "dmI_k += -2.0 * mean_I[k] * dvar;",
     "dmI_k += -mean_I[k] * dvar;"),
    ("adjoint: transposed box mean without the window counts",
     "for (int i = 0; i < w; ++i) z[(size_t)j * w + i] = y[(size_t)j * w + i] / window_count(j, i, h, w, r);",
     "for (int i = 0; i < w; ++i) z[(size_t)j * w + i] = y[(size_t)j * w + i];"),
    ("adjoint: transposed upsample off by half a pixel",
     "axis_taps((X + 0.5) / (double)s - 0.5, w, &x0, &x1, &fx);",
     "axis_taps((X + 0.5) / (double)s, w, &x0, &x1, &fx);"),
    ("adjoint: transposed bilinear subsample with a wrong weight",
     "x[(size_t)y0 * W + x1] += (1.0 - fy) * fx * g;",
     "x[(size_t)y0 * W + x1] += (1.0 - fy) * (1.0 - fx) * g;"),
    ("colour guide: eps tripled on the diagonal (R12)",
     "M[k][k] += eps;",
     "M[k][k] += 3.0 * eps;"),
    ("colour guide: wrong sign of b (R12)",
     "bb -= x[k] * mean_I[k * n + t];",
     "bb += x[k] * mean_I[k * n + t];"),
    ("colour guide: covariance matrix filled on one side only (R12)",
     "M[PL[m]][PK[m]] = e;",
     "M[PL[m]][PK[m]] = 0.5 * e;"),
    ("depthwise guide: every channel guided by guide channel 0 (R8)",
     "const double *Ig = I + ((size_t)bn * CI + (CI == 1 ? 0 : c)) * NF;\n            /* step 1",
     "const double *Ig = I + ((size_t)bn * CI + 0) * NF;\n            /* step 1"),
    ("adjoint: depthwise guide channel 0 for every channel",
     "const double *Ig = I + ((size_t)bn * CI + (CI == 1 ? 0 : c)) * NF;\n            const double *g = gq",
     "const double *Ig = I + ((size_t)bn * CI + 0) * NF;\n            const double *g = gq"),
    ("adjoint: wrong sign of d eps",
     "eps_acc += dvar;",
     "eps_acc -= dvar;"),
    ("adjoint: transposed upsample off by half a row",
     "axis_taps((Yi + 0.5) / (double)s - 0.5, h, &y0, &y1, &fy);",
     "axis_taps((Yi + 0.5) / (double)s, h, &y0, &y1, &fy);"),
    ("adjoint: transposed nearest subsample without the half-pixel offset",
     "int sy = iclamp((int)floor((j + 0.5) * s), 0, H - 1);",
     "int sy = iclamp((int)floor(j * (double)s), 0, H - 1);"),
    ("adjoint: gradient of a low-res p dropped",
     "memcpy(dpc, dpl, sizeof(double) * n);",
     "memset(dpc, 0, sizeof(double) * n);"),
    ("Algorithm 1: summed-area window one column short",
     "int ia = imax(0, i - r), ib = imin(w - 1, i + r) + 1;",
     "int ia = imax(0, i - r), ib = imin(w - 1, i + r) + (r > 0 ? 0 : 1);"),
    ("colour guide: guide products squared instead of crossed (R12)",
     "for (size_t t = 0; t < n; ++t) tmp[t] = Il[PK[m] * n + t] * Il[PL[m] * n + t];",
     "for (size_t t = 0; t < n; ++t) tmp[t] = Il[PK[m] * n + t] * Il[PK[m] * n + t];"),
    ("non-integer ratio: bilinear subsample offset ignoring the denominator (R13)",
     "axis_taps_q((2LL * i + 1) * sn - sd, 2LL * sd, W, &x0, &x1, &fx);",
     "axis_taps_q((2LL * i + 1) * sn - 1, 2LL * sd, W, &x0, &x1, &fx);"),
    ("non-integer ratio: upsample scale with the denominator dropped (R13)",
     "axis_taps_q((2LL * Y + 1) * sd - sn, 2LL * sn, h, &y0, &y1, &fy);",
     "axis_taps_q((2LL * Y + 1) - sn / sd, 2LL * (sn / sd), h, &y0, &y1, &fy);"),
    ("non-integer ratio: low-res width from the integer part of s (R13)",
     "*w = (int)(((long long)W * sd + sn - 1) / sn);",
     "*w = (int)(((long long)W + sn / sd - 1) / (sn / sd));"),
    ("low-res p of image 0 for every image of a batch (Alg. 2)",
     "memcpy(pl, p + ((size_t)bn * C + c) * n, sizeof(double) * n);\n            else\n                gfo_subsample_q(",
     "memcpy(pl, p + ((size_t)c) * n, sizeof(double) * n);\n            else\n                gfo_subsample_q("),
    ("adjoint: low-res p of image 0 for every image of a batch",
     "memcpy(pl, p + ((size_t)bn * C + c) * n, sizeof(double) * n);\n            else\n                "
     "gfo_subsample(p + ((size_t)bn * C + c) * NF, H, W, s, mode, pl);\n            box_mean_mode",
     "memcpy(pl, p + ((size_t)c) * n, sizeof(double) * n);\n            else\n                "
     "gfo_subsample(p + ((size_t)bn * C + c) * NF, H, W, s, mode, pl);\n            box_mean_mode"),
    ("colour guide: low-res p of image 0 for every image of a batch (R12)",
     "memcpy(pl, p + ((size_t)bn * C + c) * n, sizeof(double) * n);\n            else\n                "
     "gfo_subsample(p + ((size_t)bn * C + c) * NF, H, W, s, mode, pl);\n            gfo_box_mean(pl",
     "memcpy(pl, p + ((size_t)c) * n, sizeof(double) * n);\n            else\n                "
     "gfo_subsample(p + ((size_t)bn * C + c) * NF, H, W, s, mode, pl);\n            gfo_box_mean(pl"),
    ("box sum one column short (R1)",
     "for (int ii = imax(0, i - r); ii <= imin(w - 1, i + r); ++ii) acc += x[(size_t)j * w + ii];",
     "for (int ii = imax(0, i - r); ii < imin(w - 1, i + r); ++ii) acc += x[(size_t)j * w + ii];"),
    ("antialiased subsample without renormalising the weights (R11)",
     "v = acc / wsum;",
     "v = acc;"),
    ("adjoint: direct term g U(mean_a) of dI dropped",
     "for (size_t k = 0; k < NF; ++k) dIg[k] += g[k] * up_a[k];",
     "for (size_t k = 0; k < NF; ++k) dIg[k] += 0.0 * g[k] * up_a[k];"),
    ("adjoint: p' term of dI' dropped",
     "dIl[k] += 2.0 * Il[k] * tI[k] + pl[k] * tp[k];",
     "dIl[k] += 2.0 * Il[k] * tI[k];"),
    ("colour guide: wrong sign in the 3 x 3 determinant (R12)",
     "- M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])",
     "+ M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])"),
    ("detail epilogue: guide channel 0 for every channel (Fig. 2)",
     "const double *Ic = I + ((size_t)n * CI + (CI == 1 ? 0 : c)) * HW;",
     "const double *Ic = I + ((size_t)n * CI + 0) * HW;"),
    ("window count unclipped along the rows (R1)",
     "int nx = imin(w - 1, i + r) - imax(0, i - r) + 1;",
     "int nx = 2 * r + 1;"),
    ("brute-force box mean divided by the full window (R1)",
     "y[(size_t)j * w + i] = acc / (double)n;",
     "y[(size_t)j * w + i] = acc / (double)((2 * r + 1) * (2 * r + 1));"),
    ("r' not raised to 1 for small r (R6)",
     "if (r >= 1 && rl < 1) rl = 1;",
     "if (r >= 1 && rl < 0) rl = 1;"),
    ("adjoint: eps left out of the derivative of a",
     "double inv = 1.0 / (var[k] + eps);",
     "double inv = 1.0 / (var[k] + 0.5 * eps);"),
    ("adjoint: brute-force transposed box mean without the window counts",
     "double v = y[(size_t)j * w + i] / window_count(j, i, h, w, r);",
     "double v = y[(size_t)j * w + i];"),
    ("colour guide: box means of a skipped (R12)",
     "for (int k = 0; k < 3; ++k) gfo_box_mean(a + k * n, h, w, r_low, mean_a + k * n);",
     "for (int k = 0; k < 3; ++k) memcpy(mean_a + k * n, a + k * n, sizeof(double) * n);"),
    ("antialiased subsample over too narrow a span of source pixels (R11)",
     "int span = 3 * ((sn + sd - 1) / sd) + 3;",
     "int span = (sn + sd - 1) / sd;"),
    ("Algorithm 1: wrong sign of b",
     "b[k] = mp[k] - a[k] * mI[k];",
     "b[k] = mp[k] + a[k] * mI[k];"),
    ("adjoint: d a missing the path through b",
     "double da_k = da[k] - mean_I[k] * db[k];",
     "double da_k = da[k];"),
    ("adjoint: d mean_p missing the path through cov",
     "dmp_k += -mean_I[k] * dcov;",
     "dmp_k += 0.0 * dcov;"),
    ("adjoint: transposed box subsample dividing ragged blocks by s^2",
     "double v = g / (double)((yb - ya) * (xb - xa));",
     "double v = g / (double)(s * s);"),
    ("detail epilogue with the detail layer reversed (Fig. 2)",
     "oc[i] = qc[i] + k * (Ic[i] - qc[i]);",
     "oc[i] = qc[i] + k * (qc[i] - Ic[i]);"),
]


def _build_copy(name, text):
    os.makedirs(OUT, exist_ok=True)
    stem = "".join(ch if ch.isalnum() else "_" for ch in name)[:48] + "_%08x" % zlib.crc32(name.encode())
    src, lib = os.path.join(OUT, stem + ".c"), os.path.join(OUT, stem + ".so")
    with open(src, "w") as f:
        f.write(text)
    oracle.compile_library(src, lib)
    return lib


def _failing_pins(lib):
    failed = []
    with oracle.use_library(lib):
        for name, pin in PINS:
            try:
                pin()
            except Exception:  # an assertion, or the planted build rejecting its arguments
                failed.append(name)
    return failed


def test_unmodified_copy_passes_every_pin():
    lib = _build_copy("unmodified", open(SRC).read())
    assert _failing_pins(lib) == []


@pytest.mark.parametrize("name,anchor,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(name, anchor, planted):
    text = open(SRC).read()
    assert text.count(anchor) == 1, "the text to replace must occur exactly once"
    lib = _build_copy(name, text.replace(anchor, planted))
    assert _failing_pins(lib), "no pin catches: " + name
