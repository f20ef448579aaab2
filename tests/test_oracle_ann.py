"""Pins for the oracle's 3D PatchMatch (Sec. 3.1, Algorithm 1): validity of
the shift map, monotone distances, the exhaustive nearest neighbour, the scan
directions of the printed (sequential) algorithm, the random-search radius
r_max rho^k (Eq. 3); and for the two options beside it: the original
PatchMatch multi-radius search (every r_max rho^i >= 1 per iteration) and
several propagation sub-sweeps per iteration."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_05528_gb300 import synth


def _setup(seed=0, W=24, H=20, T=12, C=3):
    rng = np.random.default_rng(seed)
    x = synth.smooth_noise(rng, H, W, 2.0, channels=C).astype(np.float32)
    x = np.repeat(x[None], T, axis=0)
    x = x + 0.05 * rng.random((T, H, W, C), dtype=np.float32)
    hole = np.zeros((T, H, W), np.uint8)
    hole[4:8, 7:12, 9:15] = 1
    ht, dt = O.masks(hole)
    phi = O.init_nnf(ht, dt, (1, 2), O.tag(O.PURPOSE_INIT, 0))
    return np.ascontiguousarray(x, dtype=np.float32), hole, ht, dt, phi


def _valid(phi, target, dtilde):
    tt, yy, xx = np.nonzero(target)
    st = tt + phi[tt, yy, xx, 2]
    sy = yy + phi[tt, yy, xx, 1]
    sx = xx + phi[tt, yy, xx, 0]
    T, H, W = target.shape
    inb = (st >= 0) & (st < T) & (sy >= 0) & (sy < H) & (sx >= 0) & (sx < W)
    return inb.all() and (dtilde[st, sy, sx] == 1).all()


@pytest.mark.parametrize("schedule", ["SEQ", "JAC"])
def test_shift_map_stays_valid_and_distances_non_increasing(schedule):
    x, hole, ht, dt, phi0 = _setup()
    prev = None
    key = (7, 8)
    for n_pm in range(0, 7):
        phi = phi0.copy()
        d2 = np.full(hole.shape, np.inf, np.float32)
        O.ann(x, ht, dt, phi, d2, n_pm=n_pm, schedule=schedule, key=key,
              tag_base=O.tag(O.PURPOSE_SEARCH, 0, 0))
        assert _valid(phi, ht, dt)
        assert np.isfinite(d2[ht == 1]).all()
        if prev is not None:
            # iteration n_pm continues iteration n_pm - 1 (same draws)
            assert (d2[ht == 1] <= prev[ht == 1]).all()
        prev = d2.copy()
        # stored distances are those of the stored shifts (FP32 definition)
        for (t, y, xx) in list(zip(*np.nonzero(ht)))[::37]:
            s = (xx + phi[t, y, xx, 0], y + phi[t, y, xx, 1], t + phi[t, y, xx, 2])
            assert d2[t, y, xx] == O.dist(x, (xx, y, t), s)


def test_energy_non_increasing_with_fixed_video():
    x, hole, ht, dt, phi = _setup(seed=3)
    d2 = np.full(hole.shape, np.inf, np.float32)
    e0 = O.energy(x, hole, ht, phi)
    O.ann(x, ht, dt, phi, d2, n_pm=10, key=(1, 1))
    e1 = O.energy(x, hole, ht, phi)
    assert e1[0] <= e0[0] and e1[1] <= e0[1]


@pytest.mark.parametrize("schedule", ["SEQ", "JAC"])
def test_never_below_exhaustive_nn(schedule):
    x, hole, ht, dt, phi = _setup(seed=1, W=18, H=16, T=9)
    d2 = np.full(hole.shape, np.inf, np.float32)
    O.ann(x, ht, dt, phi, d2, n_pm=10, schedule=schedule, key=(3, 3))
    bphi, bd2 = O.bruteforce_nn(x, ht, dt)
    m = ht == 1
    assert (d2[m] >= bd2[m]).all()
    # the search gets close on this easy volume
    assert np.mean(d2[m]) <= 3.0 * np.mean(bd2[m]) + 1e-4


def test_exhaustive_nn_is_a_fixed_point():
    # starting from the exact nearest neighbours, no candidate is strictly
    # better: Algorithm 1 returns them unchanged
    x, hole, ht, dt, _ = _setup(seed=2, W=18, H=16, T=9)
    bphi, bd2 = O.bruteforce_nn(x, ht, dt)
    phi = bphi.copy()
    d2 = np.full(hole.shape, np.inf, np.float32)
    O.ann(x, ht, dt, phi, d2, n_pm=6, key=(9, 9))
    np.testing.assert_array_equal(phi[ht == 1], bphi[ht == 1])
    np.testing.assert_array_equal(d2[ht == 1], bd2[ht == 1])


def _translation_row_case():
    # u(x, y, t) = f(x - t, y): the shift (c, 0, c) is an exact match. A row of
    # targets at y = 8, t = 6, x = 10..21; the leftmost holds the true shift
    # (d = 0), the others a bad shift. rmax = 0 turns the random search into a
    # no-op (its candidate is p + phi(p) itself), isolating the propagation.
    W, H, T = 40, 16, 16
    x = synth.translating_texture(W, H, T, sigma=1.5, seed=77)
    hole = np.zeros((T, H, W), np.uint8)
    _, dt = O.masks(hole)
    target = np.zeros((T, H, W), np.uint8)
    xs = list(range(10, 22))
    target[6, 8, xs] = 1
    phi = np.zeros((T, H, W, 3), np.int32)
    phi[6, 8, xs] = (-6, 4, 2)          # a valid, non-matching shift
    phi[6, 8, xs[0]] = (4, 0, 4)        # true shift: (14, 8, 10) matches exactly
    return x, target, dt, phi, xs


def test_sequential_scan_direction_and_in_place_update():
    # Algorithm 1: k = 1 is odd (reverse scan, +1 neighbours), k = 2 even
    # (forward scan, -1 neighbours) and updates in place, so the true shift
    # travels along the whole row during sweep k = 2.
    x, target, dt, phi, xs = _translation_row_case()
    d2 = np.full(target.shape, np.inf, np.float32)
    O.ann(x, target, dt, phi, d2, n_pm=1, schedule="SEQ", rmax=0)
    assert d2[6, 8, xs[0]] == 0.0 and (d2[6, 8, xs[1:]] > 0).all()
    O.ann(x, target, dt, phi, d2, n_pm=2, schedule="SEQ", rmax=0)
    assert (d2[6, 8, xs] == 0.0).all()
    assert (phi[6, 8, xs] == (4, 0, 4)).all()


def test_jacobi_schedule_moves_one_voxel_per_sweep():
    # the parallel schedule reads the shifts of the start of the sweep: after
    # k = 1, 2 only the right-hand neighbour of the seed has it; after
    # k = 1..4 two of them (k = 2 and k = 4 are the forward sweeps).
    x, target, dt, phi0, xs = _translation_row_case()
    for n_pm, n_good in [(1, 1), (2, 2), (3, 2), (4, 3), (6, 4)]:
        phi = phi0.copy()
        d2 = np.full(target.shape, np.inf, np.float32)
        O.ann(x, target, dt, phi, d2, n_pm=n_pm, schedule="JAC", rmax=0)
        assert (d2[6, 8, xs] == 0.0).sum() == n_good, n_pm


def test_random_search_radius():
    # A flat video where every source is an exact match except the one the
    # targets start on: each valid random candidate is accepted, so after one
    # iteration (k = 1) phi - phi0 = floor(r_max rho^1 delta) for accepted
    # targets, which spans [-r_max/2, r_max/2 - 1] and no more.
    W, H, T = 64, 64, 64
    x = np.full((T, H, W, 1), 0.5, np.float32)
    x[30:35, 30:35, 30:35, 0] = 0.9        # the bad source patch at (32, 32, 32)
    hole = np.zeros((T, H, W), np.uint8)
    _, dt = O.masks(hole)
    target = np.zeros((T, H, W), np.uint8)
    target[8:56:2, 8:56:2, 8:56:2] = 1     # isolated targets: no propagation
    tt, yy, xx = np.nonzero(target)
    phi = np.zeros((T, H, W, 3), np.int32)
    phi[tt, yy, xx, 0] = 32 - xx
    phi[tt, yy, xx, 1] = 32 - yy
    phi[tt, yy, xx, 2] = 32 - tt
    phi0 = phi.copy()
    d2 = np.full(target.shape, np.inf, np.float32)
    rmax = 40
    O.ann(x, target, dt, phi, d2, n_pm=1, schedule="JAC", rmax=rmax, key=(5, 6))
    moved = (phi[tt, yy, xx] != phi0[tt, yy, xx]).any(axis=1)
    off = (phi - phi0)[tt, yy, xx][moved]
    assert moved.mean() > 0.5
    assert off.min() == -rmax // 2 and off.max() == rmax // 2 - 1
    # with rho = 0.25 the first radius is r_max / 4
    phi = phi0.copy()
    O.ann(x, target, dt, phi, d2, n_pm=1, schedule="JAC", rmax=rmax, rho=0.25, key=(5, 6))
    off = (phi - phi0)[tt, yy, xx]
    assert off.min() == -rmax // 4 and off.max() == rmax // 4 - 1


def test_random_search_is_schedule_independent():
    # with no target adjacent to another, the propagation never fires and SEQ
    # and JAC must agree bit for bit
    x, hole, ht, dt, phi0 = _setup(seed=4)
    iso = np.zeros_like(ht)
    iso[::2, ::2, ::2] = ht[::2, ::2, ::2]
    a, b = phi0.copy(), phi0.copy()
    da = np.full(hole.shape, np.inf, np.float32)
    db = da.copy()
    O.ann(x, iso, dt, a, da, n_pm=10, schedule="SEQ", key=(4, 4))
    O.ann(x, iso, dt, b, db, n_pm=10, schedule="JAC", key=(4, 4))
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(da, db)


def test_jacobi_sub_sweeps_spread_one_voxel_each():
    # J propagation sweeps per iteration k: during each forward iteration
    # (k even) the seed's shift travels J voxels, during k odd none (the row's
    # seed is its leftmost voxel)
    x, target, dt, phi0, xs = _translation_row_case()
    for n_pm, J in [(2, 1), (2, 3), (4, 2), (3, 4), (4, 5)]:
        phi = phi0.copy()
        d2 = np.full(target.shape, np.inf, np.float32)
        O.ann(x, target, dt, phi, d2, n_pm=n_pm, schedule="JAC", rmax=0, sub_sweeps=J)
        want = min(1 + J * (n_pm // 2), len(xs))
        assert (d2[6, 8, xs] == 0.0).sum() == want, (n_pm, J)


def _flat_case():
    W, H, T = 64, 64, 64
    x = np.full((T, H, W, 1), 0.5, np.float32)
    x[30:35, 30:35, 30:35, 0] = 0.9        # the bad source patch at (32, 32, 32)
    hole = np.zeros((T, H, W), np.uint8)
    _, dt = O.masks(hole)
    target = np.zeros((T, H, W), np.uint8)
    target[8:56:2, 8:56:2, 8:56:2] = 1     # isolated targets: no propagation
    tt, yy, xx = np.nonzero(target)
    phi = np.zeros((T, H, W, 3), np.int32)
    phi[tt, yy, xx, 0] = 32 - xx
    phi[tt, yy, xx, 1] = 32 - yy
    phi[tt, yy, xx, 2] = 32 - tt
    return x, target, dt, phi, (tt, yy, xx)


def test_multi_radius_search_starts_at_r_max():
    # the original PatchMatch search tries r_max rho^i for i = 0, 1, ...: its
    # first candidate (accepted whenever valid and clear of the bad patch, as
    # almost every source matches exactly) moves the shift by
    # floor(r_max delta), spanning [-r_max, r_max - 1]
    # (r_max = 24 keeps every first candidate inside D~: sources 32 +- 24)
    x, target, dt, phi0, (tt, yy, xx) = _flat_case()
    phi = phi0.copy()
    d2 = np.full(target.shape, np.inf, np.float32)
    rmax = 24
    O.ann(x, target, dt, phi, d2, n_pm=1, schedule="JAC", rmax=rmax, key=(5, 6), rs_mode=1)
    off = (phi - phi0)[tt, yy, xx]
    moved = (off != 0).any(axis=1)
    assert moved.mean() > 0.9
    assert off.min() == -rmax and off.max() == rmax - 1


def test_multi_radius_search_counts_every_radius():
    # isolated targets whose every candidate is valid make one evaluation per
    # radius r_max 2^-i >= 1 per iteration (plus the initial distance): with
    # r_max = 8, radii 8, 4, 2, 1
    x, target, dt, phi0, (tt, yy, xx) = _flat_case()
    one = np.zeros_like(target)
    one[32, 32, 32] = 1
    phi = np.zeros_like(phi0)
    d2 = np.full(target.shape, np.inf, np.float32)
    ev = O.ann(x, one, dt, phi, d2, n_pm=3, schedule="JAC", rmax=8, key=(1, 1), rs_mode=1)
    assert ev == 1 + 3 * 4
    ev = O.ann(x, one, dt, phi, d2, n_pm=3, schedule="JAC", rmax=8, key=(1, 1), rs_mode=0)
    assert ev == 1 + 3 * 1


def test_multi_radius_with_one_radius_matches_eq3():
    # r_max = 1: the multi-radius search has the single radius 1, drawn from
    # counter word 3 = 0, which is Eq. 3's candidate at k = 1 with r_max = 2
    x, hole, ht, dt, phi0 = _setup(seed=6)
    a, b = phi0.copy(), phi0.copy()
    da = np.full(hole.shape, np.inf, np.float32)
    db = da.copy()
    ea = O.ann(x, ht, dt, a, da, n_pm=1, schedule="JAC", rmax=1, key=(3, 3), rs_mode=1)
    eb = O.ann(x, ht, dt, b, db, n_pm=1, schedule="JAC", rmax=2, key=(3, 3), rs_mode=0)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(da, db)
    assert ea == eb


@pytest.mark.parametrize("schedule", ["SEQ", "JAC"])
def test_multi_radius_and_sub_sweeps_keep_validity_and_monotonicity(schedule):
    x, hole, ht, dt, phi = _setup(seed=8)
    d2 = np.full(hole.shape, np.inf, np.float32)
    O.ann(x, ht, dt, phi, d2, n_pm=0)
    prev = d2.copy()
    for call in range(3):
        O.ann(x, ht, dt, phi, d2, n_pm=4, schedule=schedule, key=(2, 3), tag_base=call,
              rs_mode=1, sub_sweeps=2)
        assert _valid(phi, ht, dt)
        assert (d2[ht == 1] <= prev[ht == 1]).all()
        prev = d2.copy()


@pytest.mark.parametrize("rs_mode,sub_sweeps", [(0, 1), (1, 1), (0, 2)])
def test_rescore_then_iterations_is_the_jacobi_search(rs_mode, sub_sweeps):
    # rescore followed by ann_iteration for k = 1 .. n_pm (the split the rank
    # harness of the time slabs exchanges between) is ann's Jacobi schedule
    x, hole, ht, dt, phi0 = _setup(seed=9)
    a, b = phi0.copy(), phi0.copy()
    da = np.full(hole.shape, np.inf, np.float32)
    db = da.copy()
    ea = O.ann(x, ht, dt, a, da, n_pm=5, schedule="JAC", key=(4, 1), tag_base=77, rs_mode=rs_mode,
               sub_sweeps=sub_sweeps)
    eb = O.rescore(x, ht, dt, b, db)
    for k in range(1, 6):
        eb += O.ann_iteration(x, ht, dt, b, db, k, key=(4, 1), tag_base=77, rs_mode=rs_mode,
                              sub_sweeps=sub_sweeps)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(da.view(np.uint32), db.view(np.uint32))
    assert ea == eb
