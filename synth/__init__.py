"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This package holds input recipes only (scenes, noise, quantisation, request streams).  It contains none
of the filter's arithmetic, so both the GPU path and the oracle can be fed from it.
"""
from .scenes import (  # noqa: F401
    make_scene, rgb_noisy_input, quantize_u8, to_f16_values, trainable_layer_batch, serving_stream,
    block_mean_downsample, make_color_scene, feather_mask,
)
