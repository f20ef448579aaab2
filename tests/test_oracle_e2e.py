"""Pins for the oracle's initialisation (Algorithm 3) and complete method
(Algorithm 4): convexity of the onion-peel filling, its layer structure, the
translation special case with a planted exact shift, and the parallel
schedule's energy against the printed sequential one."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_05528_gb300 import synth


def test_onion_peel_fills_every_hole_voxel_convexly():
    c = synth.small_layered(W=48, H=40, T=10, levels=1, seed=21)
    pyr = O.build_pyramid(c.rgb, c.mask, 1, use_texture=True)
    lv = pyr[0]
    prm = O.Params()
    lv.phi = O.init_nnf(lv.htilde, lv.dtilde, prm.key, O.tag(O.PURPOSE_INIT, 0))
    lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
    x_before = lv.x.copy()
    n = O.onion_peel(lv, prm, 0)
    assert n >= 2
    hole = lv.hole.astype(bool)
    known = x_before[~hole]
    # every filled value is a convex combination of known values (Eq. 12)
    for ch in range(lv.x.shape[-1]):
        v = lv.x[hole][:, ch]
        assert v.min() >= known[:, ch].min() - 1e-6
        assert v.max() <= known[:, ch].max() + 1e-6
    np.testing.assert_array_equal(lv.x[~hole], x_before[~hole])


def test_onion_layers_of_a_box():
    # a 7x7x5 interior box: layers are the successive 3x3x3 erosions, so the
    # count is the box's half-thickness in its thinnest direction (t: 5 -> 3)
    W, H, T = 30, 30, 13
    rgb = synth.translating_texture(W, H, T, seed=3)
    mask = synth.box_mask(W, H, T, 12, 18, 12, 18, 4, 8)
    pyr = O.build_pyramid(rgb, mask, 1, use_texture=False)
    lv = pyr[0]
    prm = O.Params()
    lv.phi = O.init_nnf(lv.htilde, lv.dtilde, prm.key, 0)
    lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
    assert O.onion_peel(lv, prm, 0) == 3


def test_onion_peel_hole_touching_the_volume_border():
    # a tube through every frame: its faces on the first and last frame have
    # no known neighbour in t; their interior voxels wait (deferred) until the
    # lateral peeling reaches them, and every voxel is filled in the end
    W, H, T = 32, 32, 8
    rgb = synth.translating_texture(W, H, T, seed=4)
    mask = synth.box_mask(W, H, T, 12, 19, 12, 19, 0, T - 1)
    pyr = O.build_pyramid(rgb, mask, 1, use_texture=False)
    lv = pyr[0]
    prm = O.Params()
    lv.phi = O.init_nnf(lv.htilde, lv.dtilde, prm.key, 0)
    lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
    n = O.onion_peel(lv, prm, 0)
    assert n >= 4
    assert np.isfinite(lv.x).all()


def _translation_case():
    # translation special case: u(x, y, t) = f(x - 4t, y) on 48x48x16 with a
    # 4x4x2 hole; the shift (4c, 0, c) maps every patch onto an identical one,
    # and (12, 0, 3) reaches sources clear of the hole for every target.
    W, H, T = 48, 48, 16
    rgb = synth.translating_texture(W, H, T, sigma=2.0, seed=9, speed=4)
    mask = synth.box_mask(W, H, T, 22, 25, 22, 25, 7, 8)
    return rgb, mask


def test_planted_true_shift_reconstructs_exactly():
    rgb, mask = _translation_case()
    pyr = O.build_pyramid(rgb, mask, 1, use_texture=False)
    lv = pyr[0]
    T, H, W = mask.shape
    phi = np.zeros((T, H, W, 3), np.int32)
    phi[...] = (12, 0, 3)
    tt, yy, xx = np.nonzero(lv.htilde)
    st, sx = tt + 3, xx + 12
    assert (lv.dtilde[st, yy, sx] == 1).all()
    d2 = np.full(mask.shape, np.inf, np.float32)
    lv.phi = phi
    lv.d2 = d2
    # the known part of every target patch is an exact copy, the hole is 0:
    # one vote with exact shifts returns the ground truth
    O.ann(lv.x, lv.htilde, lv.dtilde, lv.phi, lv.d2, n_pm=0)
    out, _ = O.vote(lv.x, lv.hole, lv.htilde, lv.phi, lv.d2, weighted=True)
    np.testing.assert_allclose(out[mask == 1], rgb[mask == 1], atol=1e-6)
    # and then the energy of the planted state is 0
    assert O.energy(out, lv.hole, lv.htilde, lv.phi) == (0.0, 0.0)


@pytest.mark.slow
def test_full_run_translation_case():
    rgb, mask = _translation_case()
    out, pyr, before = O.inpaint(rgb, mask, 1, use_texture=False,
                                 prm=O.Params(fixed_outer=10), return_levels=True)
    lv = pyr[0]
    eh, _ = O.energy(before, lv.hole, lv.htilde, lv.phi)
    err = out[mask == 1] - rgb[mask == 1]
    psnr = 10 * np.log10(1.0 / max(float(np.mean(err ** 2)), 1e-20))
    assert eh / mask.sum() < 2e-3
    assert psnr > 30.0
    np.testing.assert_array_equal(out[mask == 0], rgb[mask == 0])


def test_jacobi_energy_close_to_sequential_tiny_clip():
    c = synth.tiny_translation_clip()
    es = {}
    for sched in ("SEQ", "JAC"):
        prm = O.Params(schedule=sched, fixed_outer=10)
        out, pyr, before = O.inpaint(c.rgb, c.mask, 1, use_texture=False, prm=prm,
                                     return_levels=True)
        lv = pyr[0]
        es[sched] = O.energy(before, lv.hole, lv.htilde, lv.phi)[0]
        assert np.isfinite(out).all()
    assert abs(es["JAC"] - es["SEQ"]) <= 0.02 * es["SEQ"]


@pytest.mark.slow
def test_multilevel_with_texture_runs():
    c = synth.small_layered(W=64, H=48, T=12, levels=2, seed=31)
    prm = O.Params(fixed_outer=[3, 2])
    out, pyr, before = O.inpaint(c.rgb, c.mask, 2, use_texture=True, prm=prm,
                                 return_levels=True)
    assert np.isfinite(out).all()
    assert pyr[1].stats["onion_layers"] >= 1
    assert pyr[0].stats["outer"] == [2] and pyr[1].stats["outer"] == [3]


def test_iteration_cap_counts_from_call_zero():
    # Sec. 3.7's cap of max_outer iterations per level counts the level's
    # iterations from call 0: a loop resumed at call start_call runs at most
    # max_outer - start_call more
    from paper_1503_05528_gb300 import synth as S
    c = S.small_layered(W=40, H=32, T=10, levels=1, seed=1903)
    lv = O.build_pyramid(c.rgb, c.mask, 1, True)[0]
    lv.phi = O.init_nnf(lv.htilde, lv.dtilde, (1, 1), O.tag(O.PURPOSE_INIT, 0))
    lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
    prm = O.Params(seed=5, stop=0.0, max_outer=4)      # stop 0: only the cap ends the loop
    assert O.iterate_level(lv, prm, 0, start_call=2) == 2
    assert O.iterate_level(lv, prm, 0, start_call=4) == 0


def test_white_noise_hole_is_filled_smoother_than_the_noise():
    # The toy example of Appendix B (Fig. 11): in i.i.d. noise no source patch
    # is much closer than another, so the weighted mean of Eq. 4 averages many
    # unrelated noise samples and the hole comes out smoother than the noise
    # around it; the best-patch step (Eq. 6) copies single noise voxels back.
    rng = np.random.default_rng(21)
    T, H, W = 8, 28, 28
    rgb = np.clip(0.5 + 0.1 * rng.standard_normal((T, H, W, 3)), 0.0, 1.0).astype(np.float32)
    mask = np.zeros((T, H, W), np.uint8)
    mask[2:6, 10:18, 10:18] = 1
    prm = O.Params(seed=4, fixed_outer=[6])
    out, pyr, before = O.inpaint(rgb, mask, 1, use_texture=False, prm=prm, return_levels=True)
    h = mask == 1
    noise = rgb[~h].std()
    assert before[h][:, :3].std() < 0.6 * noise
    assert out[h].std() > 0.8 * noise     # Eq. 6 copies noise voxels
