"""Pins for three parts of the oracle's level loop that no other test fixes:
the stopping value e of Sec. 3.7, the split of Eq. 1 into E_H and E_H~, and
the provisional fill of the level transition (Sec. 3.6).

The first two use a clip whose source set D~ holds exactly one patch. Every
target's shift then has to point at that patch (a propagated shift lands
elsewhere, and a random candidate is valid only when it equals the current
shift), so the search cannot change the shift map and every distance, vote
and stopping value has a closed form written out below by hand."""
import numpy as np
import pytest

from oracle import oracle as O

W, H, T = 8, 5, 5
HOLE = [(5, 2, 2), (6, 2, 2)]   # (x, y, t)
SRC = (2, 2, 2)                  # the one centre whose patch is whole and misses H
# channel c of voxel (x, y, t) is A[c] * x + B[c] outside the hole
A = np.array([0.1, -0.05, 0.02, 0.3, -0.2])
B = np.array([0.1, 0.6, 0.3, 0.0, 0.5])


def _ramp_level(hole_values=None):
    xs = np.arange(W, dtype=np.float64)
    x = np.empty((T, H, W, 5), np.float32)
    for c in range(5):
        x[..., c] = (A[c] * xs + B[c])[None, None, :]
    hole = np.zeros((T, H, W), np.uint8)
    for i, (hx, hy, ht) in enumerate(HOLE):
        hole[ht, hy, hx] = 1
        if hole_values is not None:
            x[ht, hy, hx] = hole_values[i]
    ht_, dt_ = O.masks(hole)
    lv = O.Level(x, hole, ht_, dt_)
    return lv


def _n_in(c, n):
    """Voxels of [c - 2, c + 2] inside [0, n)."""
    return min(c + 2, n - 1) - max(c - 2, 0) + 1


def test_single_source_clip_has_the_closed_form_sets():
    lv = _ramp_level()
    assert lv.dtilde.sum() == 1 and lv.dtilde[SRC[2], SRC[1], SRC[0]] == 1
    # H~: every voxel within 2 of a hole voxel in x, y and t
    want = np.zeros((T, H, W), np.uint8)
    want[:, :, 3:8] = 1
    np.testing.assert_array_equal(lv.htilde, want)


def test_energy_splits_into_hole_and_target_sums():
    # Eq. 1 over H and the same sum over H~. On the ramp (hole values on the
    # ramp too) a target p matched to the single source s has
    #   d^2(p) = n_in(p) / 125 * sum_c A_c^2 * (p_x - s_x)^2,
    # n_in(p) the voxels of its patch inside the video (Eq. 2 divides by 125).
    hv = [A * hx + B for (hx, _, _) in HOLE]
    lv = _ramp_level(hv)
    phi = np.zeros((T, H, W, 3), np.int32)
    tt, yy, xx = np.nonzero(lv.htilde)
    phi[tt, yy, xx, 0] = SRC[0] - xx
    phi[tt, yy, xx, 1] = SRC[1] - yy
    phi[tt, yy, xx, 2] = SRC[2] - tt
    a2 = float((A ** 2).sum())
    e_h = 0.0
    for (hx, hy, ht) in HOLE:
        e_h += _n_in(hx, W) * _n_in(hy, H) * _n_in(ht, T) / 125.0 * a2 * (hx - SRC[0]) ** 2
    e_ht = 0.0
    for (t, y, x) in zip(tt, yy, xx):
        e_ht += _n_in(x, W) * _n_in(y, H) * _n_in(t, T) / 125.0 * a2 * (x - SRC[0]) ** 2
    # by hand: the hole voxels give 9 a2 (x = 5, all 125 in) + 12.8 a2 (x = 6,
    # 100 in); H~ gives (19 * 19 / 125) * 209 a2
    assert e_h == pytest.approx(21.8 * a2, rel=1e-12)
    assert e_ht == pytest.approx(361.0 / 125.0 * 209.0 * a2, rel=1e-12)
    got_h, got_ht = O.energy(lv.x, lv.hole, lv.htilde, phi)
    assert got_h == pytest.approx(e_h, rel=1e-6)
    assert got_ht == pytest.approx(e_ht, rel=1e-6)


def test_stopping_value_counts_rgb_change_over_three_hole_voxels():
    # e of Sec. 3.7 after one iteration of the level loop: the mean absolute
    # change of R, G, B over the occluded voxels, sum / (3 |H|). The
    # unweighted vote (Eq. 4 with s = 1) averages x(p + phi(q)) = x(s + p - q)
    # over the targets q of N_p: at x = 5 the offsets p_x - q_x are -2..2
    # (mean 0), at x = 6 they are -1..2 (q_x <= 7; mean 0.5), so on the ramp
    # the new values are A * 2 + B and A * 2.5 + B. The old values differ in
    # both directions, and the texture channels change a lot, which e must
    # not count.
    old = [np.array([0.9, 0.0, 0.5, 5.0, -3.0]), np.array([0.0, 0.9, 0.1, 7.0, 2.0])]
    lv = _ramp_level(old)
    prm = O.Params(weighted=False, seed=5)
    lv.phi = O.init_nnf(lv.htilde, lv.dtilde, prm.key, O.tag(O.PURPOSE_INIT, 0))
    lv.d2 = np.full(lv.hole.shape, np.inf, np.float32)
    O.iterate_level(lv, prm, 0, n_outer=1)
    new = [A * 2.0 + B, A * 2.5 + B]
    for (hx, hy, ht), v in zip(HOLE, new):
        np.testing.assert_allclose(lv.x[ht, hy, hx], v.astype(np.float32), atol=2e-7)
    # the shift map is still the forced one
    tt, yy, xx = np.nonzero(lv.htilde)
    assert (lv.phi[tt, yy, xx, 0] == SRC[0] - xx).all()
    # |0.3 - 0.9| + |0.5 - 0| + |0.34 - 0.5| + |0.35 - 0| + |0.475 - 0.9| + |0.35 - 0.1|
    change = sum(float(np.abs(n[:3] - o[:3]).sum()) for n, o in zip(new, old))
    assert change == pytest.approx(2.285, abs=1e-12)
    e = lv.stats["e"][-1]
    assert e == pytest.approx(2.285 / 6.0, rel=1e-6)
    # the mistakes this excludes give other values: all five channels,
    # |H~| = 125 instead of |H|, or signed changes
    assert abs(e - sum(float(np.abs(n - o).sum()) for n, o in zip(new, old)) / 6.0) > 1.0
    assert abs(e - 2.285 / (3 * 125)) > 0.3
    assert abs(e - sum(float((n[:3] - o[:3]).sum()) for n, o in zip(new, old)) / 6.0) > 0.1


def _parent_fill_by_hand(coarse_x, fine_x, fine_hole, tsub):
    out = fine_x.copy()
    Tf, Hf, Wf = fine_hole.shape
    for t in range(Tf):
        for y in range(Hf):
            for x in range(Wf):
                if fine_hole[t, y, x]:
                    out[t, y, x] = coarse_x[t // 2 if tsub else t, y // 2, x // 2]
    return out


@pytest.mark.parametrize("tsub", [False, True])
def test_provisional_fill_takes_the_coarse_parent(tsub):
    # every coarse voxel holds a distinct value, so a wrong parent index
    # (no halving in y, x and y swapped, t halved or not) picks another one
    rng = np.random.default_rng(11)
    Tc = 4 if tsub else 7
    Tf = 7
    coarse = rng.random((Tc, 6, 7, 5)).astype(np.float32)
    fine = rng.random((Tf, 12, 13, 5)).astype(np.float32)
    hole = np.zeros((Tf, 12, 13), np.uint8)
    hole[2:5, 3:10, 4:11] = 1          # odd and even x, y, t
    want = _parent_fill_by_hand(coarse, fine, hole, tsub)
    got = O.provisional_fill(coarse, fine.copy(), hole, tsub)
    np.testing.assert_array_equal(got, want)
    # one odd voxel spelled out
    assert (got[3, 5, 7] == coarse[1 if tsub else 3, 2, 3]).all()


def test_transition_distances_are_taken_on_the_parent_filled_video():
    # The level transition re-scores the upsampled shifts on the video whose
    # occluded voxels hold their coarse parents' values, and votes afterwards.
    # The distances it leaves must equal distances computed on a fill done by
    # hand (the vote reads only known voxels and does not change them).
    from paper_1503_05528_gb300 import synth
    c = synth.small_layered(W=40, H=32, T=8, levels=2, seed=9)
    prm = O.Params(seed=3)
    pyr = O.build_pyramid(c.rgb, c.mask, 2, use_texture=True)
    coarse, fine = pyr[1], pyr[0]
    coarse.phi = O.init_nnf(coarse.htilde, coarse.dtilde, prm.key, O.tag(O.PURPOSE_INIT, 1))
    coarse.d2 = np.full(coarse.hole.shape, np.inf, np.float32)
    # a coarse video that varies in x, y and t inside the hole too
    rng = np.random.default_rng(4)
    coarse.x = (coarse.x + 0.1 * rng.random(coarse.x.shape)).astype(np.float32)
    filled = _parent_fill_by_hand(coarse.x, fine.x, fine.hole, False)
    O.next_level(coarse, fine, prm, 0)
    tt, yy, xx = np.nonzero(fine.htilde)
    assert len(tt) > 100
    for (t, y, x) in zip(tt, yy, xx):
        dx, dy, dt = fine.phi[t, y, x]
        want = O.dist(filled, (x, y, t), (x + dx, y + dy, t + dt))
        assert fine.d2[t, y, x] == want
