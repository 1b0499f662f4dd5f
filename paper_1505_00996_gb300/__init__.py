"""GB300-native (sm_103a) fast guided filter: He and Sun, "Fast Guided Filter" (arXiv:1505.00996).

The compute path is ``libgf.so`` (hand-written CUDA kernels behind the C ABI of ``include/gf.h``); this
package is a thin ctypes binding over it that uses PyTorch for device memory and streams.
"""
from .binding import (  # noqa: F401
    GF_OK, GF_PENDING, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ETIMEOUT, GF_EBUSY, GF_ECANCELED, GF_ENOTFOUND, GF_EWAIT,
    GF_SUB_NEAREST, GF_SUB_BILINEAR, GF_SUB_BOX, GF_SUB_BILINEAR_AA, GF_F32, GF_F16, GF_U8, GF_MAX_STAGES, MODES,
    GFError, GFOpts, Context, default_context, fast_guided_filter, fast_guided_filter_host, load_library,
    library_path, lowres_geometry, opts_init, fast_guided_filter_backward, row_band, row_strips, host_strips,
    kernel_faults, backward_workspace_size,
)
from .autograd import FastGuidedFilter, FastGuidedFilterFn  # noqa: F401
from .serving import Server  # noqa: F401
