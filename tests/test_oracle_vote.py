"""Pins for the oracle's reconstruction (Eq. 4/5, Eq. 9, Eq. 12) and final
best-patch step (Eq. 6): hand-computed weighted means, the sigma = 0 limit,
the closed form of Appendix A (the unweighted mean minimises the energy for a
fixed shift map) and special cases."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _line_case(values, d2s, shifts, W):
    """A 1-row, 1-frame volume; voxel 0 is voted from its in-volume
    neighbours q = 0..len(d2s)-1 (the patch is clipped by the video)."""
    x = np.zeros((1, 1, W, 1), np.float32)
    for i, v in enumerate(values):
        x[0, 0, i, 0] = v
    phi = np.zeros((1, 1, W, 3), np.int32)
    d2 = np.zeros((1, 1, W), np.float32)
    for q, (s, d) in enumerate(zip(shifts, d2s)):
        phi[0, 0, q, 0] = s
        d2[0, 0, q] = d
    vote = np.zeros((1, 1, W), np.uint8)
    vote[0, 0, 0] = 1
    allowed = np.ones((1, 1, W), np.uint8)
    return x, vote, allowed, phi, d2


def test_weighted_vote_three_contributors():
    # p = voxel 0 of a 4-voxel line: N_p in the video = {0, 1, 2}. q = 0, 1, 2
    # point at voxels 1, 2, 3 (values 0.2, 0.6, 1.0) with d^2 = 0.01, 0.04, 0.09.
    # The 75th percentile (nearest rank ceil(0.75*3) = 3rd) is sigma^2 = 0.09,
    # so s = exp(-0.01/0.18), exp(-0.04/0.18), exp(-0.09/0.18).
    x, vote, allowed, phi, d2 = _line_case([0.0, 0.2, 0.6, 1.0], [0.01, 0.04, 0.09], [1, 2, 3], 4)
    s = [math.exp(-1 / 18), math.exp(-2 / 9), math.exp(-0.5)]
    want = (0.2 * s[0] + 0.6 * s[1] + 1.0 * s[2]) / sum(s)
    out, _ = O.vote(x, vote, allowed, phi, d2, weighted=True, n_diff=1)
    assert out[0, 0, 0, 0] == pytest.approx(want, abs=2e-7)
    assert want == pytest.approx(0.54231, abs=1e-5)


def test_weighted_vote_rank_of_percentile():
    # 2x2 frame corner: N_p = 4 voxels, d^2 = (0.01, 0.02, 0.05, 0.5):
    # nearest rank ceil(0.75*4) = 3 gives sigma^2 = 0.05 (not an interpolated
    # value between 0.05 and 0.5).
    x = np.zeros((1, 3, 3, 1), np.float32)
    vals = {(0, 0): 0.0, (0, 2): 0.1, (1, 2): 0.3, (2, 0): 0.5, (2, 2): 0.9}
    for (y, xx), v in vals.items():
        x[0, y, xx, 0] = v
    phi = np.zeros((1, 3, 3, 3), np.int32)
    d2 = np.zeros((1, 3, 3), np.float32)
    # q at (0,0),(1,0),(0,1),(1,1) (x, y); p + phi(q) lands on the value cells
    spec = {(0, 0): ((2, 0), 0.01), (1, 0): ((2, 1), 0.02), (0, 1): ((0, 2), 0.05),
            (1, 1): ((2, 2), 0.5)}
    for (qx, qy), ((tx, ty), d) in spec.items():
        phi[0, qy, qx] = (tx, ty, 0)        # p = (0, 0), so p + phi(q) = (tx, ty)
        d2[0, qy, qx] = d
    vote = np.zeros((1, 3, 3), np.uint8)
    vote[0, 0, 0] = 1
    # keep the contributors to the 4 voxels of the 2x2 corner
    allowed = np.zeros((1, 3, 3), np.uint8)
    allowed[0, 0:2, 0:2] = 1
    out, _ = O.vote(x, vote, allowed, phi, d2, weighted=True, n_diff=1)
    w = [math.exp(-0.01 / 0.1), math.exp(-0.02 / 0.1), math.exp(-0.05 / 0.1), math.exp(-0.5 / 0.1)]
    v = [0.1, 0.3, 0.5, 0.9]
    want = sum(a * b for a, b in zip(w, v)) / sum(w)
    assert out[0, 0, 0, 0] == pytest.approx(want, abs=2e-7)
    # unweighted: the plain mean
    out, _ = O.vote(x, vote, allowed, phi, d2, weighted=False, n_diff=1)
    assert out[0, 0, 0, 0] == pytest.approx(sum(v) / 4, abs=1e-7)


def test_sigma_zero_limit():
    # three of four distances are 0: sigma^2 = 0 and only the exact matches
    # vote (the limit of exp(-d^2 / 2 sigma^2) as sigma -> 0)
    x, vote, allowed, phi, d2 = _line_case([0.0, 0.2, 0.6, 1.0, 0.3], [0.0, 0.0, 0.0],
                                           [1, 2, 3], 5)
    d2[0, 0, 0:3] = [0.0, 0.0, 0.0]
    # a 1-D line with 5 voxels: N_p = {0,1,2}; make q = 2 a non-match
    d2[0, 0, 2] = 0.3
    out, _ = O.vote(x, vote, allowed, phi, d2, weighted=True, n_diff=1)
    # ranks: sorted (0, 0, 0.3), ceil(2.25) = 3rd -> sigma^2 = 0.3 > 0 here
    s = [1.0, math.exp(-0.0), math.exp(-0.5)]
    want = (0.2 * s[0] + 0.6 * s[1] + 1.0 * s[2]) / sum(s)
    assert out[0, 0, 0, 0] == pytest.approx(want, abs=2e-7)
    # now 4 contributors (2-D corner) with three zeros: sigma^2 = 0
    x2 = np.zeros((1, 3, 3, 1), np.float32)
    x2[0, 2, 2, 0] = 0.9
    x2[0, 2, 1, 0] = 0.4
    phi2 = np.zeros((1, 3, 3, 3), np.int32)
    d22 = np.zeros((1, 3, 3), np.float32)
    phi2[0, 0, 0] = (2, 2, 0)
    phi2[0, 0, 1] = (1, 2, 0)
    phi2[0, 1, 0] = (1, 2, 0)
    phi2[0, 1, 1] = (2, 2, 0)
    d22[0, 1, 1] = 0.7
    vote2 = np.zeros((1, 3, 3), np.uint8)
    vote2[0, 0, 0] = 1
    allowed2 = np.zeros((1, 3, 3), np.uint8)
    allowed2[0, 0:2, 0:2] = 1
    out2, _ = O.vote(x2, vote2, allowed2, phi2, d22, weighted=True, n_diff=1)
    assert out2[0, 0, 0, 0] == pytest.approx((0.9 + 0.4 + 0.4) / 3, abs=1e-7)


def _random_state(seed=0, W=22, H=18, T=10, C=3):
    rng = np.random.default_rng(seed)
    x = rng.random((T, H, W, C), dtype=np.float32)
    hole = np.zeros((T, H, W), np.uint8)
    hole[3:7, 6:11, 8:14] = 1
    ht, dt = O.masks(hole)
    phi = O.init_nnf(ht, dt, (seed, 1), 0)
    d2 = np.full(hole.shape, np.inf, np.float32)
    O.ann(x, ht, dt, phi, d2, n_pm=2, key=(seed, 2))
    return x, hole, ht, dt, phi, d2


def test_unweighted_vote_minimises_energy_appendix_a():
    # Appendix A: for a fixed shift map, E over H~ is a sum of independent
    # quadratics in the u(p), p in H, minimised by the plain mean of the
    # u(p + phi(q)). The vote must lower E and be a stationary minimum.
    x, hole, ht, dt, phi, d2 = _random_state(1)
    e_before = O.energy(x, hole, ht, phi)[1]
    out, _ = O.vote(x, hole, ht, phi, d2, weighted=False, n_diff=3)
    e_after = O.energy(out, hole, ht, phi)[1]
    assert e_after <= e_before
    rng = np.random.default_rng(7)
    tt, yy, xx = np.nonzero(hole)
    for i in rng.choice(len(tt), 6, replace=False):
        for c in range(3):
            for eps in (+2e-3, -2e-3):
                pert = out.copy()
                pert[tt[i], yy[i], xx[i], c] += eps
                assert O.energy(pert, hole, ht, phi)[1] > e_after


def test_vote_reads_only_known_voxels():
    # Sec. 2: p + phi(q) lies in the patch of q + phi(q) in D~, hence in D.
    # Changing the values of occluded voxels must not change the vote.
    x, hole, ht, dt, phi, d2 = _random_state(2)
    a, _ = O.vote(x, hole, ht, phi, d2, weighted=True)
    x2 = x.copy()
    x2[hole == 1] = 123.0
    b, _ = O.vote(x2, hole, ht, phi, d2, weighted=True)
    np.testing.assert_array_equal(a[hole == 1], b[hole == 1])


def test_constant_shift_copies_source():
    x, hole, ht, dt, _, _ = _random_state(3)
    T, H, W = hole.shape
    phi = np.zeros((T, H, W, 3), np.int32)
    phi[...] = (-7, 0, 0)
    rng = np.random.default_rng(0)
    d2 = rng.random(hole.shape).astype(np.float32)
    out, _ = O.vote(x, hole, ht, phi, d2, weighted=True)
    tt, yy, xx = np.nonzero(hole)
    np.testing.assert_allclose(out[tt, yy, xx], x[tt, yy, xx - 7], rtol=0, atol=1e-7)


def test_final_best_patch_eq6():
    x, hole, ht, dt, phi, d2 = _random_state(4)
    out = O.final(x, hole, phi, d2)
    T, H, W = hole.shape
    for (t, y, xx) in list(zip(*np.nonzero(hole)))[::11]:
        # the argmin over q in N_p, first in (dt, dy, dx) order
        best, bq = np.inf, None
        for a in range(-2, 3):
            for b in range(-2, 3):
                for c in range(-2, 3):
                    q = (t + a, y + b, xx + c)
                    if 0 <= q[0] < T and 0 <= q[1] < H and 0 <= q[2] < W and d2[q] < best:
                        best, bq = d2[q], q
        s = (t + phi[bq][2], y + phi[bq][1], xx + phi[bq][0])
        np.testing.assert_array_equal(out[t, y, xx], x[s])
    # known voxels are untouched
    np.testing.assert_array_equal(out[hole == 0], x[hole == 0])


def test_final_ties_take_first_in_patch_order():
    x, hole, ht, dt, phi, _ = _random_state(5)
    d2 = np.ones(hole.shape, np.float32)     # all equal: q* = p + (-2, -2, -2) when inside
    out = O.final(x, hole, phi, d2)
    t, y, xx = [int(v[0]) for v in np.nonzero(hole)]
    q = (t - 2, y - 2, xx - 2)
    s = (q[0] + phi[q][2] + 2, q[1] + phi[q][1] + 2, q[2] + phi[q][0] + 2)
    np.testing.assert_array_equal(out[t, y, xx], x[s])


def test_deferred_when_no_contributor():
    x, hole, ht, dt, phi, d2 = _random_state(6)
    allowed = np.zeros_like(hole)
    out, ch, deferred = O.vote(x, hole, allowed, phi, d2, want_deferred=True)
    assert (deferred == hole).all() and ch == 0.0
    np.testing.assert_array_equal(out, x)
