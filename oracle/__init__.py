"""FP64 CPU oracle for the Fast Guided Filter (He and Sun, 2015).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library (``paper_1505_00996_gb300``) never imports it, and
the two share no code.  See ``gf_oracle.c`` for the readings of the paper's open points (R1-R13).
"""
from .oracle import (  # noqa: F401
    SUB_NEAREST, SUB_BILINEAR, SUB_BOX, SUB_BILINEAR_AA, build, lowres_radius, lowres_shape, subsample, box_sum, box_mean,
    box_mean_bruteforce, upsample, fast_guided_filter, guided_filter, fast_guided_filter_backward,
    detail_enhance, color_guided_filter, ratio, compile_library, use_library,
)
