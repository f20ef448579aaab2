"""The seeded synthetic workloads that stand in for the paper's videos (the
recipe of each, checked on the CPU): sizes, occlusion fractions and
structure as stated, values in range, known voxels untouched by the mask,
and the same clip for the same seed."""
import numpy as np

from paper_1503_05528_gb300 import synth


def test_tiny_clip_is_a_translating_texture_with_a_centred_box():
    c = synth.tiny_translation_clip()
    assert c.rgb.shape == (8, 32, 32, 3) and c.mask.shape == (8, 32, 32)
    assert c.mask.sum() == 8 * 8 * 4
    assert c.mask[2:6, 12:20, 12:20].all()
    # u(x, y, t) = f(x - t, y): frame t is frame 0 shifted by t (periodic)
    for t in range(8):
        np.testing.assert_array_equal(c.rgb[t], np.roll(c.rgb[0], t, axis=1))
    assert c.rgb.min() >= 0.1 - 1e-6 and c.rgb.max() <= 0.9 + 1e-6


def test_layered_clip_occlusion_fraction_and_determinism():
    a = synth.layered_clip(96, 64, 20, 2, (10, 20), 0.08, 3, 2101)
    b = synth.layered_clip(96, 64, 20, 2, (10, 20), 0.08, 3, 2101)
    np.testing.assert_array_equal(a.rgb, b.rgb)
    np.testing.assert_array_equal(a.mask, b.mask)
    assert abs(a.mask.mean() - 0.08) < 0.01
    assert a.rgb.dtype == np.float32 and a.mask.dtype == np.uint8
    assert np.isfinite(a.rgb).all() and a.rgb.min() >= 0.0 and a.rgb.max() <= 1.0
    # the tube is present in every frame and moves
    per_frame = a.mask.reshape(20, -1).sum(axis=1)
    assert (per_frame > 0).all()
    assert not np.array_equal(a.mask[0], a.mask[-1])


def test_workload_size_distributions():
    for (lo_w, hi_w, lo_h, hi_h, lo_t, hi_t, lo_f, hi_f), sizes in (
            ((160, 640, 120, 480, 20, 80, 0.03, 0.12), synth.batch_sizes()),
            ((320, 1280, 240, 720, 30, 120, 0.03, 0.10), synth.serve_sizes())):
        a = np.array(sizes)
        W, H, T, f = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
        assert (W >= lo_w).all() and (W <= hi_w).all() and (W % 2 == 0).all()
        assert (H >= lo_h).all() and (H <= hi_h).all() and (H % 2 == 0).all()
        assert (T >= lo_t).all() and (T <= hi_t).all() and (T % 2 == 0).all()
        assert (f >= lo_f).all() and (f <= hi_f).all()
        # log-uniform: the median near the geometric mean of the bounds
        assert abs(np.log(np.median(W)) - 0.5 * np.log(lo_w * hi_w)) < 0.35
    assert len(synth.batch_sizes()) == 48 and len(synth.serve_sizes()) == 200
    assert synth.batch_sizes() == synth.batch_sizes()
