"""Pins for the oracle's random draws: Philox4x32-10 against its published
known-answer vectors, the word -> (-1, 1) and word -> index maps, and the
shift-map initialisation / upsampling (Sec. 3.1, Sec. 3.6)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(v, 16) for v in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expected", _kat())
def test_philox_known_answers(ctr, key, expected):
    assert list(O.philox4x32_10(ctr, key)) == expected


def test_philox_counter_sensitivity():
    base = O.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert list(O.philox4x32_10(c, [5, 6])) != list(base)


def test_unit_symmetric_range_and_symmetry():
    lo = O.unit_symmetric(0)
    hi = O.unit_symmetric(0xFFFFFFFF)
    assert lo == -1.0 + 2.0 ** -24
    assert hi == 1.0 - 2.0 ** -24
    # the map is odd around the middle: w and its bitwise complement give -delta
    for w in [0, 255, 256, 12345678, 0x7FFFFFFF, 0x80000000, 0xDEADBEEF]:
        assert O.unit_symmetric(w) == -O.unit_symmetric(0xFFFFFFFF ^ w)
    # mean of many draws is ~0 and the spread is that of U(-1,1)
    vals = np.array([O.unit_symmetric(int(O.philox4x32_10([i, 7, 0, 0], [1, 2])[0]))
                     for i in range(4000)])
    assert abs(vals.mean()) < 0.05
    assert abs(vals.var() - 1.0 / 3.0) < 0.03


def test_uniform_index_bounds_and_uniformity():
    assert O.uniform_index(0, 17) == 0
    assert O.uniform_index(0xFFFFFFFF, 17) == 16
    n = 10
    counts = np.zeros(n)
    for i in range(5000):
        counts[O.uniform_index(int(O.philox4x32_10([i, 1, 0, 0], [3, 4])[0]), n)] += 1
    exp = 5000 / n
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 30.0   # 9 dof; p ~ 4e-4


def _hole_and_sets(W=24, H=20, T=10):
    hole = np.zeros((T, H, W), np.uint8)
    hole[3:7, 6:12, 8:15] = 1
    ht, dt = O.masks(hole)
    return hole, ht, dt


def test_init_nnf_valid_and_uniform():
    hole, ht, dt = _hole_and_sets()
    phi = O.init_nnf(ht, dt, (11, 12), O.tag(O.PURPOSE_INIT, 0))
    T, H, W = hole.shape
    tt, yy, xx = np.nonzero(ht)
    st = tt + phi[tt, yy, xx, 2]
    sy = yy + phi[tt, yy, xx, 1]
    sx = xx + phi[tt, yy, xx, 0]
    assert (dt[st, sy, sx] == 1).all()
    # uniform over D~: the empirical source histogram over time slices is flat
    n_src_t = dt.sum(axis=(1, 2)).astype(float)
    got = np.bincount(st, minlength=T).astype(float)
    expv = len(st) * n_src_t / n_src_t.sum()
    m = expv > 0
    chi2 = ((got[m] - expv[m]) ** 2 / expv[m]).sum()
    assert chi2 < 3 * m.sum() + 20
    # non-target voxels untouched
    assert (phi[ht == 0] == 0).all()


def test_upsample_constant_shift_doubles():
    # coarse level: a constant shift everywhere; fine level: spatial x2 size
    Wc, Hc, T = 20, 16, 10
    Wf, Hf = 40, 32
    hole_f = np.zeros((T, Hf, Wf), np.uint8)
    hole_f[4:6, 14:18, 18:22] = 1
    ht_f, dt_f = O.masks(hole_f)
    phi_c = np.zeros((T, Hc, Wc, 3), np.int32)
    phi_c[..., 0] = -5
    phi_c[..., 1] = 3
    phi_c[..., 2] = 1
    phi_f = O.upsample_nnf(phi_c, ht_f, dt_f, (1, 2), O.tag(O.PURPOSE_UPSAMPLE, 0))
    tt, yy, xx = np.nonzero(ht_f)
    sx, sy, st = xx - 10, yy + 6, tt + 1
    ok = ((sx >= 0) & (sx < Wf) & (sy >= 0) & (sy < Hf) & (st >= 0) & (st < T))
    ok[ok] &= dt_f[st[ok], sy[ok], sx[ok]] == 1
    got = phi_f[tt, yy, xx]
    assert ok.any() and (~ok).any()
    assert (got[ok] == np.array([-10, 6, 1])).all()
    # the others were redrawn into D~
    bx = xx[~ok] + got[~ok, 0]
    by = yy[~ok] + got[~ok, 1]
    bt = tt[~ok] + got[~ok, 2]
    assert (dt_f[bt, by, bx] == 1).all()


def test_upsample_reads_parent():
    # every coarse voxel holds a distinct shift; fine voxel (x, y, t) must take
    # the one of (x//2, y//2, t)
    Wc, Hc, T = 12, 12, 8
    Wf, Hf = 24, 24
    hole_f = np.zeros((T, Hf, Wf), np.uint8)
    hole_f[3:5, 10:14, 10:14] = 1
    ht_f, _ = O.masks(hole_f)
    dt_all = np.ones((T, Hf, Wf), np.uint8)   # every shift is accepted
    rng = np.random.default_rng(3)
    phi_c = rng.integers(-3, 4, size=(T, Hc, Wc, 3)).astype(np.int32)
    phi_f = O.upsample_nnf(phi_c, ht_f, dt_all, (1, 2), 0)
    for (t, y, x) in zip(*np.nonzero(ht_f)):
        want = phi_c[t, y // 2, x // 2] * np.array([2, 2, 1])
        sx, sy, st = x + want[0], y + want[1], t + want[2]
        if 0 <= sx < Wf and 0 <= sy < Hf and 0 <= st < T:
            assert (phi_f[t, y, x] == want).all()
