"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, exports every function that
include/gf.h declares, and its host-only entry points (defaults, geometry, workspace size, argument
checks) behave as documented.  No kernel is launched here."""
import ctypes
import os
import re
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1505_00996_gb300 import _build, binding
    _build.build_library()
    return binding.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gf_create", "gf_destroy", "gf_filter", "gf_filter_host", "gf_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lib, n)


def test_opts_defaults(lib):
    from paper_1505_00996_gb300 import binding
    o = binding.opts_init()
    assert (o.batch, o.guide_channels, o.r_low, o.p_lowres, o.dtype_in, o.dtype_out) == (1, 1, -1, 0, 0, 0)
    assert not o.workspace and not o.kernel_events
    assert lib.gf_abi_version() == 5
    assert o.saved_forward == 0 and o.test_wait_fault == 0


@pytest.mark.parametrize("H,W,s,r", [(3000, 4000, 4, 16), (3000, 4000, 8, 16), (3000, 4000, 1, 16), (10, 13, 4, 6),
                                     (7, 7, 8, 3), (512, 512, 4, 8), (1, 1, 3, 0)])
def test_lowres_geometry_matches_oracle_rule(lib, H, W, s, r):
    from paper_1505_00996_gb300 import binding
    h, w, rp = binding.lowres_geometry(H, W, s, r)
    assert (h, w) == oracle.lowres_shape(H, W, s)
    assert rp == oracle.lowres_radius(r, s)
    assert binding.lowres_geometry(H, W, s, r, r_low=5)[2] == 5


def test_workspace_size(lib):
    from paper_1505_00996_gb300 import binding
    o = binding.opts_init()
    n = ctypes.c_size_t()
    binding.check(lib.gf_workspace_size(3000, 4000, 3, 4, ctypes.byref(o), ctypes.byref(n)))
    # low-res 750 x 1000: I', 3 x p', 3 x (a, b, mean_a, mean_b) planes of FP32
    assert n.value >= (1 + 3 + 12) * 750 * 1000 * 4
    n1 = ctypes.c_size_t()
    binding.check(lib.gf_workspace_size(3000, 4000, 3, 1, ctypes.byref(o), ctypes.byref(n1)))
    assert n1.value >= 12 * 3000 * 4000 * 4


def test_argument_errors_are_reported_without_launching(lib):
    from paper_1505_00996_gb300 import binding
    o = binding.opts_init()
    n = ctypes.c_size_t()
    assert lib.gf_workspace_size(0, 10, 1, 4, ctypes.byref(o), ctypes.byref(n)) == binding.GF_EINVAL
    assert b"H, W and C" in lib.gf_last_error()
    assert lib.gf_workspace_size(10, 10, 1, 0, ctypes.byref(o), ctypes.byref(n)) == binding.GF_EINVAL
    o.guide_channels = 2
    assert lib.gf_workspace_size(10, 10, 3, 2, ctypes.byref(o), ctypes.byref(n)) == binding.GF_EINVAL
    o = binding.opts_init()
    o.dtype_in = binding.GF_U8
    o.r_low = 40  # (2*40+1)^2 * 1020^2 > 2^32 at s = 4 bilinear
    assert lib.gf_workspace_size(400, 400, 1, 4, ctypes.byref(o), ctypes.byref(n)) == binding.GF_EINVAL
    assert lib.gf_filter(None, None, None, None, 8, 8, 1, 1, 0.1, 1, 1, None, None) == binding.GF_EINVAL
    assert lib.gf_lowres_geometry(0, 1, 1, 1, -1, None, None, None) == binding.GF_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1505_00996_gb300 import _build, binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(_build, "LIB_PATH", str(tmp_path / "missing" / "libgf.so"))
    with pytest.raises(RuntimeError):
        binding.load_library(build_if_missing=False)


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1505_00996_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "gf_oracle" not in text and "libgforacle" not in text, f


def test_kernel_count(lib, monkeypatch):
    from paper_1505_00996_gb300 import binding
    o = binding.opts_init()
    count = lambda H, W, s, mode: lib.gf_filter_kernel_count(H, W, 3, s, mode, ctypes.byref(o))
    assert count(3000, 4000, 4, binding.GF_SUB_BILINEAR) == 4
    # s = 1: no subsample stage, and the identity upsample lets the box means of a, b and the output share
    # one kernel (rows a multiple of 4 pixels); otherwise statistics, box means and output apart
    assert count(3000, 4000, 1, binding.GF_SUB_BILINEAR) == 2
    assert count(3000, 4001, 1, binding.GF_SUB_BILINEAR) == 3
    assert count(0, 4000, 4, binding.GF_SUB_BILINEAR) == -1
    # the subsample and the statistics as one kernel: opt-in, at r' = 4 (given through opts.r_low)
    o.r_low = 4
    assert count(3000, 4000, 4, binding.GF_SUB_BILINEAR) == 4
    monkeypatch.setenv("GF_SUB_STRIP", "1")
    assert count(3000, 4000, 4, binding.GF_SUB_BILINEAR) == 3
    assert count(3000, 4000, 8, binding.GF_SUB_NEAREST) == 3
    assert count(3000, 4000, 2, binding.GF_SUB_BILINEAR) == 4  # s = 2: not taken
    o.r_low = 3
    assert count(3000, 4000, 4, binding.GF_SUB_BILINEAR) == 4  # r' = 3: not taken
    monkeypatch.delenv("GF_SUB_STRIP")


def test_automatic_single_kernel_weighs_the_halo(lib):
    """gf_opts.fused = 0 takes the single kernel while N C H W (1 + r'/4)^2 <= 2.1 * 2^20 (and N C H W <=
    2^20): the measured crossings against the chain move to smaller images as r' grows."""
    from paper_1505_00996_gb300 import binding
    o = binding.opts_init()
    count = lambda H, W, C: lib.gf_filter_kernel_count(H, W, C, 4, binding.GF_SUB_BILINEAR, ctypes.byref(o))
    o.r_low = 1
    assert count(1024, 1024, 1) == 1 and count(480, 640, 3) == 1
    o.r_low = 2
    assert count(896, 896, 1) == 1 and count(480, 640, 3) == 1
    assert count(1024, 1024, 1) == 4
    o.r_low = 4
    assert count(640, 640, 1) == 1 and count(600, 800, 1) == 1
    assert count(768, 768, 1) == 4 and count(512, 512, 3) == 4


def test_host_strips(lib):
    """The strips gf_filter_host pipelines a large host call in: contiguous, cover every row, inner
    boundaries on multiples of 8 s, at most 8; small or unsupported forms are not pipelined."""
    import torch
    from fractions import Fraction

    from paper_1505_00996_gb300 import binding
    ys = binding.host_strips(3000, 4000, 3, 4)
    assert ys[0] == 0 and ys[-1] == 3000 and 2 <= len(ys) - 1 <= 8
    assert all(a < b for a, b in zip(ys, ys[1:]))
    assert all(y % 32 == 0 for y in ys[:-1])
    assert all(b - a >= 64 * 4 or b == 3000 for a, b in zip(ys, ys[1:]))
    ys8 = binding.host_strips(3000, 4000, 3, 8, batch=2, guide_channels=3, dtype=torch.float16)
    assert ys8[0] == 0 and ys8[-1] == 3000 and all(y % 64 == 0 for y in ys8[:-1])
    assert binding.host_strips(512, 512, 1, 4) is None          # 3 MB of host data: one piece
    assert binding.host_strips(3000, 4000, 3, Fraction(5, 2)) is None
    assert binding.host_strips(500, 40000, 3, 4) is None        # fewer than 2 x 64 s rows
    with pytest.raises(binding.GFError):
        binding.host_strips(0, 4000, 3, 4)


def test_size_limits(lib):
    """The documented size limits of gf_filter, each checked on both sides of its bound (host-only)."""
    from paper_1505_00996_gb300 import binding
    n = ctypes.c_size_t()

    def ws(H, W, C, s, **fields):
        o = binding.opts_init()
        for k, v in fields.items():
            setattr(o, k, v)
        return lib.gf_workspace_size(H, W, C, s, ctypes.byref(o), ctypes.byref(n))

    assert ws(46340, 46340, 1, 4) == binding.GF_OK           # H * W = 2147395600 < 2^31
    assert ws(46341, 46341, 1, 4) == binding.GF_EINVAL       # H * W = 2147488281 >= 2^31
    assert b"2^31" in lib.gf_last_error()
    assert ws(65535, 2, 1, 1) == binding.GF_OK               # ceil(H / s) = 65535
    assert ws(65536, 2, 1, 1) == binding.GF_EINVAL
    assert ws(262140, 2, 1, 4) == binding.GF_OK              # ceil(262140 / 4) = 65535
    assert ws(262141, 2, 1, 4) == binding.GF_EINVAL
    assert ws(8, 8, 3, 4, batch=16383) == binding.GF_OK      # batch * (1 + 3) = 65532 planes
    assert ws(8, 8, 3, 4, batch=16384) == binding.GF_EINVAL  # 65536 planes
    assert ws(64, 64, 1, 4, r_low=128) == binding.GF_OK
    assert ws(64, 64, 1, 4, r_low=129) == binding.GF_EINVAL


# Each documented argument rule of gf_opts (include/gf.h), broken once: (H, W, C, s, mode, opts fields, part of
# the message).  gf_filter_kernel_count resolves the arguments exactly as gf_filter does, host-only.
ARGUMENT_RULES = [
    (64, 64, 1, 4, "bilinear", {"batch": 0}, b"batch"),
    (64, 64, 1, 4, "bilinear", {"dtype_in": 7}, b"dtype_in"),
    (64, 64, 1, 4, "bilinear", {"dtype_out": 2}, b"dtype_out"),
    (64, 64, 3, 4, "bilinear", {"color_guide": 1, "guide_channels": 1}, b"guide_channels = 3"),
    (64, 64, 3, 4, "bilinear", {"color_guide": 1, "guide_channels": 3, "dtype_in": 2}, b"colour guide"),
    (64, 64, 1, 4, "bilinear", {"color_guide": 1, "guide_channels": 3, "detail_gain": 2.0}, b"C = 3"),
    (64, 64, 1, 4, "bilinear", {"detail_gain": float("inf")}, b"detail_gain"),
    (64, 64, 1, 4, "bilinear", {"s_num": 2, "s_den": 5}, b"ratio"),
    (64, 64, 1, 4, "box", {"s_num": 5, "s_den": 2}, b"box"),
    (64, 64, 1, 4, "bilinear", {"s_num": 5, "s_den": 2, "dtype_in": 2}, b"uint8"),
    (64, 64, 1, 4, "bilinear", {"s_num": 5, "s_den": 2, "row_begin": 0, "row_end": 8}, b"row range"),
    (64, 64, 1, 4, "box", {"dtype_in": 2}, b"uint8"),
    (64, 64, 1, 4, "bilinear_aa", {"dtype_in": 2}, b"uint8"),
    (64, 64, 1, 4, "bilinear", {"dtype_in": 2, "p_lowres": 1}, b"uint8"),
    (64, 64, 1, 4, "bilinear", {"row_begin": 10, "row_end": 10}, b"row range"),
    (64, 64, 1, 4, "bilinear", {"row_begin": 0, "row_end": 65}, b"row range"),
    (64, 64, 1, 4, "bilinear", {"r_low": 129}, b"r' > 128"),
]


@pytest.mark.parametrize("H,W,C,s,mode,fields,msg", ARGUMENT_RULES,
                         ids=["-".join("%s=%s" % kv for kv in r[5].items()) + "-" + r[4] for r in ARGUMENT_RULES])
def test_documented_argument_rules(lib, H, W, C, s, mode, fields, msg):
    from paper_1505_00996_gb300 import binding
    o = binding.opts_init()
    for k, v in fields.items():
        setattr(o, k, v)
    assert lib.gf_filter_kernel_count(H, W, C, s, binding.MODES[mode], ctypes.byref(o)) == -1
    assert msg in lib.gf_last_error(), lib.gf_last_error()
    # the same arguments without the broken rule resolve
    assert lib.gf_filter_kernel_count(H, W, C, s, binding.MODES[mode], ctypes.byref(binding.opts_init())) > 0


def test_intermediate_outputs_exclude_row_ranges_and_colour(lib):
    from paper_1505_00996_gb300 import binding
    buf = (ctypes.c_float * 16)()
    o = binding.opts_init()
    o.a_out = ctypes.addressof(buf)  # host memory: only the host-side argument check runs
    o.row_begin, o.row_end = 0, 8
    assert lib.gf_filter_kernel_count(64, 64, 1, 4, binding.GF_SUB_BILINEAR, ctypes.byref(o)) == -1
    assert b"row range" in lib.gf_last_error()
    o.row_begin = o.row_end = 0
    o.color_guide, o.guide_channels = 1, 3
    assert lib.gf_filter_kernel_count(64, 64, 3, 4, binding.GF_SUB_BILINEAR, ctypes.byref(o)) == -1
    assert b"intermediates" in lib.gf_last_error()
