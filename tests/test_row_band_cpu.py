"""The row band of a strip call (gf_row_band, host-only) against the FP64 oracle, no GPU.

A call restricted to output rows [row_begin, row_end) filters only the band of input rows that
gf_row_band reports, as if it were a whole image.  The claim checked here: the oracle run on that band
alone gives the same output rows as the oracle run on the whole image (to FP64 rounding), for every
subsample mode, ratio, radius and position of the strip -- so the band keeps every window that
reaches the strip and none of the band's own cut edges leak into it.  Also checked: the rows of p that
the host-buffer call uploads for nearest and bilinear subsampling are all the subsample reads.
"""
import numpy as np
import pytest

import oracle
from paper_1505_00996_gb300 import binding


CASES = [  # (H, W, s, r, mode, row ranges)
    (64, 40, 1, 3, oracle.SUB_BILINEAR, [(0, 1), (20, 30), (63, 64), (0, 64)]),
    (97, 36, 2, 6, oracle.SUB_NEAREST, [(0, 10), (41, 42), (50, 97), (96, 97)]),
    (120, 28, 4, 8, oracle.SUB_BILINEAR, [(0, 4), (37, 61), (60, 120), (119, 120)]),
    (130, 24, 4, 16, oracle.SUB_BOX, [(5, 6), (64, 70), (100, 130)]),
    (99, 20, 3, 9, oracle.SUB_BILINEAR, [(0, 33), (33, 66), (66, 99)]),
    (256, 16, 8, 24, oracle.SUB_BILINEAR, [(0, 100), (100, 180), (180, 256), (127, 129)]),
    (45, 30, 4, 60, oracle.SUB_BILINEAR, [(10, 20)]),  # r' = 15 windows span the whole image
    (120, 28, 4, 8, oracle.SUB_BILINEAR_AA, [(0, 4), (37, 61), (60, 120), (119, 120)]),
    (99, 20, 3, 9, oracle.SUB_BILINEAR_AA, [(0, 33), (33, 66), (66, 99)]),
    (256, 16, 8, 24, oracle.SUB_BILINEAR_AA, [(100, 180), (127, 129)]),
]


@pytest.mark.parametrize("H,W,s,r,mode,ranges", CASES)
def test_band_reproduces_whole_image_rows(H, W, s, r, mode, ranges):
    rng = np.random.default_rng(H * 7 + s)
    I = rng.uniform(0, 1, (1, 1, H, W))
    p = rng.uniform(0, 1, (1, 2, H, W))
    rl = oracle.lowres_radius(r, s)
    whole = oracle.fast_guided_filter(I, p, r, 1e-2, s, mode)
    for rb, re in ranges:
        row0, rows = binding.row_band(H, W, s, r, rb, re, mode=mode)
        assert 0 <= row0 <= rb and re <= row0 + rows <= H
        assert row0 % s == 0 and ((row0 + rows) % s == 0 or row0 + rows == H)  # whole s-row blocks
        band = oracle.fast_guided_filter(I[..., row0:row0 + rows, :], p[..., row0:row0 + rows, :], r, 1e-2, s, mode,
                                         r_low=rl)
        np.testing.assert_allclose(band[..., rb - row0:re - row0, :], whole[..., rb:re, :], rtol=0, atol=1e-12)


def test_band_with_lowres_p():
    H, W, s, rl = 128, 32, 4, 2
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 1, (1, 3, H, W))
    p = rng.uniform(0, 1, (1, 3, H // s, W // s))
    whole = oracle.fast_guided_filter(I, p, 0, 1e-2, s, oracle.SUB_BOX, r_low=rl, p_lowres=True)
    for rb, re in ((0, 16), (50, 77), (100, 128)):
        row0, rows = binding.row_band(H, W, s, 0, rb, re, r_low=rl)
        band = oracle.fast_guided_filter(I[..., row0:row0 + rows, :], p[..., row0 // s:(row0 + rows) // s, :], 0, 1e-2,
                                         s, oracle.SUB_BOX, r_low=rl, p_lowres=True)
        np.testing.assert_allclose(band[..., rb - row0:re - row0, :], whole[..., rb:re, :], rtol=0, atol=1e-12)


def test_band_is_tight_for_the_interior():
    # 2 r' low-res rows beyond the strip's tap rows, in whole s-row blocks: 12 MP, s = 4, r' = 4
    assert binding.row_band(3000, 4000, 4, 16, 0, 1500) == (0, 1536)
    assert binding.row_band(3000, 4000, 4, 16, 1500, 3000) == (1464, 1536)
    assert binding.row_band(3000, 4000, 1, 16, 1000, 1010) == (968, 74)
    assert binding.row_band(3000, 4000, 4, 16, 0, 3000) == (0, 3000)


@pytest.mark.parametrize("rb,re", [(-1, 5), (5, 5), (7, 3), (0, 3001)])
def test_invalid_row_ranges(rb, re):
    with pytest.raises(binding.GFError) as ei:
        binding.row_band(3000, 4000, 4, 16, rb, re)
    assert ei.value.status == binding.GF_EINVAL


def test_row_range_excludes_low_res_outputs():
    import ctypes
    o = binding.opts_init()
    o.row_begin, o.row_end = 0, 10
    o.a_out = 4096  # never dereferenced by a host-only call
    n = ctypes.c_size_t()
    assert binding.load_library().gf_workspace_size(100, 100, 1, 4, ctypes.byref(o), ctypes.byref(n)) == binding.GF_EINVAL


def test_row_strips_partition():
    for H, parts, align in ((3000, 2, 32), (3000, 3, 32), (10, 4, 1), (7, 8, 1), (4000, 8, 64)):
        strips = binding.row_strips(H, parts, align)
        assert len(strips) == parts and strips[0][0] == 0 and strips[-1][1] == H
        assert all(a[1] == b[0] for a, b in zip(strips, strips[1:]))
        assert all(lo <= hi for lo, hi in strips)
        assert all(lo % align == 0 for lo, _ in strips)


@pytest.mark.parametrize("mode", [oracle.SUB_NEAREST, oracle.SUB_BILINEAR])
@pytest.mark.parametrize("s", [3, 4, 5, 8])
@pytest.mark.parametrize("H", [40, 43])
def test_host_upload_rows_are_the_rows_the_subsample_reads(mode, s, H):
    """gf_filter_host uploads, for nearest and bilinear subsampling at s >= 3, only rows s j + o and
    s j + o + 1 (o = floor((s - 1) / 2)) of each whole s-row block of p, and every row of a partial last
    block.  With every other row of p set to NaN, the oracle's subsample (R2, R3) must be unchanged: those
    rows are never read, not even with weight 0."""
    W = 11
    p = np.random.default_rng(H * 10 + s).uniform(0, 1, (H, W))
    o = (s - 1) // 2
    uploaded = np.zeros(H, bool)
    for j in range(H // s):
        uploaded[s * j + o] = uploaded[s * j + o + 1] = True
    uploaded[(H // s) * s:] = True
    p_holes = p.copy()
    p_holes[~uploaded] = np.nan
    ref = oracle.subsample(p, s, mode)
    got = oracle.subsample(p_holes, s, mode)
    assert not np.isnan(got).any()
    np.testing.assert_array_equal(got, ref)
    assert uploaded.sum() < H  # the rule does leave rows out


@pytest.mark.parametrize("H,W,s,r,mode", [(3000, 4000, 4, 16, "bilinear"), (3001, 4000, 4, 16, "nearest"),
                                          (2999, 3000, 8, 60, "bilinear"), (4000, 3000, 3, 9, "box"),
                                          (2500, 3400, 5, 20, "bilinear_aa")])
def test_host_strip_bands_are_whole_blocks(H, W, s, r, mode):
    """The host pipeline uploads each strip's band after the previous strips' bands and starts its sampled
    rows of p on a block boundary, so every strip's band must start on a multiple of s and end on one (or
    at H), and the bands must reach every input row a strip reads, in order."""
    ys = binding.host_strips(H, W, 3, s, mode)
    assert ys is not None
    end = 0
    for a, b in zip(ys, ys[1:]):
        row0, rows = binding.row_band(H, W, s, r, a, b, mode=mode)
        assert row0 % s == 0 and ((row0 + rows) % s == 0 or row0 + rows == H)
        assert row0 <= a and b <= row0 + rows  # the band holds the strip's own rows
        end = max(end, row0 + rows)
    assert end == H
