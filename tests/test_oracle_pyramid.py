"""Pins for the oracle's sets (D~, H~ of Sec. 2), the 3x3x3 erosion of
Algorithm 3, the texture features (Eq. 7) and the pyramids (Eq. 8,
Algorithm 4), against brute force on tiny inputs and closed forms."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O


def _random_mask(shape, p, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(shape) < p).astype(np.uint8)


def test_sets_brute_force():
    T, H, W = 7, 8, 9
    hole = _random_mask((T, H, W), 0.03, 0)
    ht, dt = O.masks(hole)
    for t, y, x in itertools.product(range(T), range(H), range(W)):
        nb = [(t + a, y + b, x + c) for a in range(-2, 3) for b in range(-2, 3) for c in range(-2, 3)]
        inside = [(a, b, c) for (a, b, c) in nb if 0 <= a < T and 0 <= b < H and 0 <= c < W]
        # H~ = union of N_p over p in H  <=>  some hole voxel within the box
        assert ht[t, y, x] == int(any(hole[q] for q in inside))
        # D~: the whole patch inside the video and known
        assert dt[t, y, x] == int(len(inside) == 125 and not any(hole[q] for q in inside))


def test_erosion_brute_force_and_layers():
    T, H, W = 6, 7, 8
    m = _random_mask((T, H, W), 0.7, 1)
    e = O.erode3(m)
    for t, y, x in itertools.product(range(T), range(H), range(W)):
        keep = m[t, y, x] == 1
        for a, b, c in itertools.product((-1, 0, 1), repeat=3):
            q = (t + a, y + b, x + c)
            if not (0 <= q[0] < T and 0 <= q[1] < H and 0 <= q[2] < W) or m[q] == 0:
                keep = False
        assert e[t, y, x] == int(keep)
    # a cube of side 2r+1 in the interior peels in exactly r+1 layers
    cube = np.zeros((11, 11, 11), np.uint8)
    cube[2:9, 2:9, 2:9] = 1        # side 7, r = 3
    n = 0
    cur = cube
    while cur.any():
        cur = O.erode3(cur)
        n += 1
    assert n == 4


def _frames(I, T=2):
    rgb = np.repeat(I[None, :, :, None], 3, axis=-1).astype(np.float32)
    return np.repeat(rgb, T, axis=0)


def test_features_linear_ramp_exact():
    # I = a x + b y: central and one-sided differences are exact, so
    # T = (|a|, |b|) everywhere the mean has samples, for any window.
    H, W = 12, 16
    a, b = 0.02, -0.03
    yy, xx = np.mgrid[0:H, 0:W]
    I = 0.3 + a * xx + b * yy
    rgb = _frames(I)
    hole = np.zeros((2, H, W), np.uint8)
    for side in [1, 2, 8]:
        Tf = O.texture_features(rgb, hole, side)
        np.testing.assert_allclose(Tf[..., 0], abs(a), rtol=1e-5)
        np.testing.assert_allclose(Tf[..., 1], abs(b), rtol=1e-5)


def test_features_grey_level_is_channel_mean():
    H, W = 6, 10
    xx = np.arange(W, dtype=np.float64)
    rgb = np.zeros((1, H, W, 3), np.float32)
    rgb[0, :, :, 0] = 0.06 * xx     # only red varies: I = R / 3
    Tf = O.texture_features(rgb, np.zeros((1, H, W), np.uint8), 1)
    np.testing.assert_allclose(Tf[..., 0], 0.02, rtol=1e-5)
    np.testing.assert_allclose(Tf[..., 1], 0.0, atol=1e-12)


def test_features_quadratic_central_and_one_sided():
    # I = x^2 / 100: central difference (I(x+1) - I(x-1))/2 = 2x/100 inside,
    # one-sided I(1) - I(0) = 1/100 at x = 0, I(W-1) - I(W-2) = (2W-3)/100 at the end
    H, W = 4, 10
    xx = np.arange(W, dtype=np.float64)
    I = np.broadcast_to(xx ** 2 / 100.0, (H, W))
    Tf = O.texture_features(_frames(I, 1), np.zeros((1, H, W), np.uint8), 1)
    want = np.array([1.0] + [2.0 * x for x in range(1, W - 1)] + [2.0 * W - 3.0]) / 100.0
    np.testing.assert_allclose(Tf[0, 0, :, 0], want, rtol=1e-5)


def test_features_window_extent():
    # a vertical step at x = 10: |I_x| = 1/2 at x = 9 and x = 10 only. With a
    # window of side 8 (offsets -4..3) the mean over 64 samples counts those
    # two columns when x-4 <= 9 and 10 <= x+3 ... per row 8 samples.
    H, W = 20, 24
    I = np.zeros((H, W))
    I[:, 10:] = 1.0
    Tf = O.texture_features(_frames(I, 1), np.zeros((1, H, W), np.uint8), 8)
    row = 10
    for x in range(4, W - 4):
        cols = [c for c in range(x - 4, x + 4) if c in (9, 10)]
        want = len(cols) * 8 * 0.5 / 64.0
        assert Tf[0, row, x, 0] == pytest.approx(want, abs=1e-12), x


def test_features_skip_samples_touching_hole():
    # garbage under the mask must not leak: a ramp with random values in the
    # hole still gives T = |a| wherever some sample is known, 0 where none is.
    H, W = 10, 14
    a = 0.05
    xx = np.arange(W, dtype=np.float64)
    I = np.broadcast_to(0.1 + a * xx, (H, W)).copy()
    hole = np.zeros((1, H, W), np.uint8)
    hole[0, 3:7, 5:9] = 1
    rng = np.random.default_rng(0)
    I[3:7, 5:9] = rng.random((4, 4))
    Tf = O.texture_features(_frames(I, 1), hole, 2)
    tx = Tf[0, ..., 0]
    assert ((np.abs(tx - a) < 1e-6) | (tx == 0.0)).all()
    # in the middle of the hole no x-derivative sample is known (window -1..0)
    assert tx[4, 7] == 0.0
    # far from the hole the value is the ramp slope
    assert tx[0, 0] == pytest.approx(a, rel=1e-6)


def test_features_constant_video_zero():
    rgb = np.full((3, 8, 8, 3), 0.4, np.float32)
    Tf = O.texture_features(rgb, np.zeros((3, 8, 8), np.uint8), 4)
    assert (Tf == 0).all()


def test_downsample_box_mean_and_or():
    T, H, W = 2, 5, 7                       # odd sizes: ceil halving
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float32)
    x = np.zeros((T, H, W, 3), np.float32)
    x[..., 0] = 0.1 * xx
    x[..., 1] = 0.05 * yy
    x[..., 2] = 0.3
    hole = np.zeros((T, H, W), np.uint8)
    hole[1, 2, 3] = 1
    xc, hc = O.downsample(x, hole)
    assert xc.shape == (T, 3, 4, 3)
    # interior 2x2 blocks: mean of a ramp is the ramp at the block centre
    assert xc[0, 0, 0, 0] == pytest.approx(0.1 * 0.5, rel=1e-6)
    assert xc[0, 1, 2, 0] == pytest.approx(0.1 * 4.5, rel=1e-6)
    assert xc[0, 1, 2, 1] == pytest.approx(0.05 * 2.5, rel=1e-6)
    # edge blocks with one child column/row keep that child's value
    assert xc[0, 0, 3, 0] == pytest.approx(0.1 * 6.0, rel=1e-6)
    assert xc[0, 2, 0, 1] == pytest.approx(0.05 * 4.0, rel=1e-6)
    assert (xc[..., 2] == np.float32(0.3)).sum() == xc[..., 2].size - 1
    # occlusion: OR of children; that block's value is unknown (0)
    assert hc[1, 1, 1] == 1 and hc.sum() == 1
    assert (xc[1, 1, 1] == 0).all()


def test_texture_pyramid_subsampling():
    rng = np.random.default_rng(4)
    T0 = rng.random((3, 20, 24, 2))
    for lv in [1, 2, 3]:
        Hl, Wl = -(-20 // 2 ** lv), -(-24 // 2 ** lv)
        Tl = O.subsample_features(T0, lv, Wl, Hl)
        np.testing.assert_array_equal(Tl, T0[:, ::2 ** lv, ::2 ** lv, :])


def test_pyramid_known_coarse_voxels_have_known_children():
    from paper_1503_05528_gb300 import synth
    c = synth.small_layered()
    pyr = O.build_pyramid(c.rgb, c.mask, 3, True)
    for lv in range(1, 3):
        fine, coarse = pyr[lv - 1], pyr[lv]
        T, Hc, Wc = coarse.hole.shape
        for t, y, x in zip(*np.nonzero(coarse.hole == 0)):
            blk = fine.hole[t, 2 * y:2 * y + 2, 2 * x:2 * x + 2]
            assert blk.sum() == 0
        assert coarse.x.shape[-1] == 5
        assert (coarse.x[coarse.hole == 1] == 0).all()


# ---- the temporal subsampling option (Sec. 3.6, used once in the paper) ----

def test_temporal_downsample_box_mean_and_or():
    rng = np.random.default_rng(11)
    for T, H, W in [(7, 6, 5), (8, 4, 4), (1, 5, 7)]:
        x = rng.random((T, H, W, 3)).astype(np.float32)
        hole = _random_mask((T, H, W), 0.1, T)
        xc, hc = O.downsample(x, hole, tsub=True)
        assert xc.shape == ((T + 1) // 2, (H + 1) // 2, (W + 1) // 2, 3)
        for t, y, xx in itertools.product(range(xc.shape[0]), range(xc.shape[1]), range(xc.shape[2])):
            kids = [(2 * t + k, 2 * y + j, 2 * xx + i) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
            kids = [q for q in kids if q[0] < T and q[1] < H and q[2] < W]
            occl = any(hole[q] for q in kids)
            assert hc[t, y, xx] == int(occl)
            if not occl:
                want = np.mean([x[q].astype(np.float64) for q in kids], axis=0)
                np.testing.assert_allclose(xc[t, y, xx], want, rtol=0, atol=2e-7)
            else:
                assert (xc[t, y, xx] == 0).all()


def test_temporal_pyramid_sizes_constants_and_features():
    T, H, W = 9, 20, 24
    rgb = np.full((T, H, W, 3), 0.25, np.float32)
    hole = np.zeros((T, H, W), np.uint8)
    hole[3:5, 8:12, 9:14] = 1
    pyr = O.build_pyramid(rgb, hole, 3, True, tsub=True)
    assert [lv.x.shape[:3] for lv in pyr] == [(9, 20, 24), (5, 10, 12), (3, 5, 6)]
    for lv in pyr:
        known = lv.hole == 0
        assert np.allclose(lv.x[known][:, :3], 0.25) and np.allclose(lv.x[known][:, 3:], 0.0)
    # features are sampled at (2^l x, 2^l y, 2^l t) of the full-resolution field
    rng = np.random.default_rng(3)
    T0 = rng.random((T, H, W, 2))
    sub = O.subsample_features(T0, 2, 6, 5, 3, tsub=True)
    for t, y, x in itertools.product(range(3), range(5), range(6)):
        assert (sub[t, y, x] == T0[4 * t, 4 * y, 4 * x]).all()
    assert (O.subsample_features(T0, 1, 12, 10) == T0[:, ::2, ::2]).all()


def test_temporal_upsampling_doubles_all_components():
    T, H, W = 12, 16, 16
    hole = np.zeros((T, H, W), np.uint8)
    hole[5:7, 6:10, 6:10] = 1
    ht, dt = O.masks(hole)
    phic = np.zeros(((T + 1) // 2, H // 2, W // 2, 3), np.int32)
    phic[...] = (2, -1, 1)
    f = O.upsample_nnf(phic, ht, dt, (1, 1), 7, tsub=True)
    tt, yy, xx = np.nonzero(ht)
    ok = [(t, y, x) for t, y, x in zip(tt, yy, xx)
          if 0 <= t + 2 < T and 0 <= y - 2 < H and 0 <= x + 4 < W and dt[t + 2, y - 2, x + 4]]
    assert ok
    for q in ok:
        assert tuple(f[q]) == (4, -2, 2)
    # without the option dt is kept
    phic2 = np.zeros((T, H // 2, W // 2, 3), np.int32)
    phic2[...] = (2, -1, 1)
    g = O.upsample_nnf(phic2, ht, dt, (1, 1), 7)
    ok2 = [(t, y, x) for t, y, x in zip(tt, yy, xx)
           if 0 <= t + 1 < T and 0 <= y - 2 < H and 0 <= x + 4 < W and dt[t + 1, y - 2, x + 4]]
    for q in ok2:
        assert tuple(g[q]) == (4, -2, 1)


def test_temporal_option_full_run():
    from paper_1503_05528_gb300 import synth
    clip = synth.small_layered(W=48, H=40, T=12, levels=2, seed=1530)
    out = O.inpaint(clip.rgb, clip.mask, 2, True, O.Params(time_subsample=True, fixed_outer=2))
    assert np.isfinite(out).all()
    assert np.array_equal(out[clip.mask == 0], clip.rgb[clip.mask == 0])
