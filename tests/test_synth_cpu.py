"""The seeded input generators (``synth``) against the recipes their docstrings give for the stand-ins of the
paper's workloads (CPU): gradient scenes with flat rectangles and N(0, 0.05^2) noise on [0, 1], noisy
per-channel inputs, blocky feathering masks, uint8 / FP16 storage, the trainable-layer batch and the
serving request stream.  They hold none of the method's arithmetic; these checks make sure that the
inputs every parity test and benchmark uses have those shapes, value ranges, structure and determinism."""
import numpy as np
import pytest

import synth


def test_scene_recipe():
    I = synth.make_scene(300, 400, seed=0)
    assert I.shape == (300, 400) and I.dtype == np.float32
    assert I.min() >= 0.0 and I.max() <= 1.0                      # clipped to [0, 1]
    np.testing.assert_array_equal(I, synth.make_scene(300, 400, seed=0))   # seeded
    assert not np.array_equal(I, synth.make_scene(300, 400, seed=1))
    # without rectangles and noise the scene is the gradient 0.5 (x / (W - 1) + y / (H - 1))
    g = synth.make_scene(5, 9, seed=3, n_rects=0, noise_sigma=0.0)
    ys, xs = np.mgrid[0:5, 0:9]
    np.testing.assert_allclose(g, 0.5 * (xs / 8 + ys / 4), atol=1e-7)
    # the noise is N(0, 0.05^2): the difference of two noise draws over a flat, unclipped scene
    a = synth.make_scene(200, 200, seed=5, n_rects=0) - synth.make_scene(200, 200, seed=5, n_rects=0, noise_sigma=0.0)
    inner = a[50:150, 50:150]                                       # gradient near 0.5: no clipping
    assert 0.045 < inner.std() < 0.055 and abs(inner.mean()) < 0.005
    # the rectangles make piecewise-flat regions: many horizontal steps are exactly zero before the noise
    flat = synth.make_scene(200, 300, seed=2, noise_sigma=0.0)
    assert (np.diff(flat, axis=1) == 0).mean() > 0.3


def test_color_scene_and_noisy_input():
    C = synth.make_color_scene(120, 160, seed=4)
    assert C.shape == (3, 120, 160) and C.min() >= 0.0 and C.max() <= 1.0
    assert not np.array_equal(C[0], C[1])                            # a colour per rectangle
    I = synth.make_scene(100, 80, seed=0)
    p = synth.rgb_noisy_input(I, seed=1)
    assert p.shape == (3, 100, 80) and p.min() >= 0.0 and p.max() <= 1.0
    d = (p[0].astype(np.float64) - I)[(I > 0.3) & (I < 0.7)]        # away from the clip
    assert 0.09 < d.std() < 0.11                                     # N(0, 0.1^2)
    assert not np.array_equal(p[0], p[1])                            # independent per channel


def test_feather_mask_is_binary_and_blocky():
    m = synth.feather_mask(256, 320, seed=4, block=16)
    assert set(np.unique(m)) <= {0.0, 1.0} and 0.0 < m.mean() < 1.0
    cells = m.reshape(16, 16, 20, 16).transpose(0, 2, 1, 3).reshape(16, 20, 256)
    assert (cells.min(axis=2) == cells.max(axis=2)).all()            # constant on every 16 x 16 cell


def test_quantisation_recipes():
    k = np.arange(256)
    np.testing.assert_array_equal(synth.quantize_u8(k / 255.0), k)  # stored values k / 255 come back as k
    x = np.random.default_rng(0).uniform(0, 1, 1000)
    assert np.abs(synth.quantize_u8(x) - 255.0 * x).max() <= 0.5     # rounded to the nearest step
    np.testing.assert_array_equal(synth.quantize_u8(np.array([1.2, -0.1])), [255, 0])  # clamped
    h = synth.to_f16_values(np.float32(1.0 + 2 ** -11))
    assert h.dtype == np.float16 and float(h) == 1.0                 # ties to even


def test_trainable_layer_batch_recipe():
    I, p = synth.trainable_layer_batch(batch=2, channels=3, size=64, s=4)
    assert I.shape == (2, 3, 64, 64) and p.shape == (2, 3, 16, 16)
    d = p.astype(np.float64) - synth.block_mean_downsample(I, 4)
    assert 0.08 < d.std() < 0.12 and abs(d.mean()) < 0.02            # block mean + N(0, 0.1^2)
    np.testing.assert_array_equal(synth.block_mean_downsample(np.arange(16.0).reshape(4, 4), 2),
                                  [[2.5, 4.5], [10.5, 12.5]])
    with pytest.raises(ValueError):
        synth.block_mean_downsample(np.zeros((5, 4)), 2)


def test_serving_stream_recipe():
    reqs = synth.serving_stream(n_requests=512, seed=2)
    assert len(reqs) == 512
    t = np.array([r["arrival_s"] for r in reqs])
    assert (np.diff(t) > 0).all()                                    # Poisson arrivals in order
    mp = np.array([r["H"] * r["W"] / 1e6 for r in reqs])
    assert mp.min() > 0.29 and mp.max() < 24.1                       # 0.3 .. 24 MP
    aspects = {round(r["W"] / r["H"], 1) for r in reqs}
    assert aspects <= {1.3, 1.8, 1.0}                                # 4:3, 16:9, 1:1
    assert {r["C"] for r in reqs} == {1, 3} and {r["s"] for r in reqs} == {4, 8}
    assert {r["eps"] for r in reqs} == {1e-4, 1e-2}
    assert all(r["r"] == int(round(0.004 * max(r["H"], r["W"]))) for r in reqs)
    assert reqs == synth.serving_stream(n_requests=512, seed=2)      # seeded
