"""Pins for the oracle's FP64 mode (distances, stored distances and
decisions in double), the reference the FP32 path's errors are stated
against: it keeps the search's invariants, its distances are the FP64
definition of Eq. 2 / 7b for the shifts it keeps, and it differs from the
FP32 search only where FP32 rounding can decide (near-ties)."""
import numpy as np

from oracle import oracle as O
from paper_1503_05528_gb300 import synth


def _level():
    c = synth.small_layered(W=40, H=32, T=10, levels=1, seed=1531)
    lv = O.build_pyramid(c.rgb, c.mask, 1, True)[0]
    rng = np.random.default_rng(2)
    h = lv.hole.astype(bool)
    lv.x[h] = rng.random((int(h.sum()), 5), dtype=np.float32)
    phi = O.init_nnf(lv.htilde, lv.dtilde, (5, 0), O.tag(O.PURPOSE_INIT, 0))
    return lv, phi


def test_fp64_search_invariants_and_definition():
    lv, phi = _level()
    d2 = np.full(lv.hole.shape, np.inf, np.float64)
    before = None
    for call in range(3):
        O.ann(lv.x, lv.htilde, lv.dtilde, phi, d2, n_pm=4, key=(5, 0),
              tag_base=O.tag(O.PURPOSE_SEARCH, 0, call), sub_sweeps=2)
        t = lv.htilde == 1
        if before is not None:
            assert (d2[t] <= before[t]).all()       # never increases with a fixed video
        before = d2.copy()
    tt, yy, xx = np.nonzero(lv.htilde)
    for (t, y, x) in list(zip(tt, yy, xx))[::7]:
        dx, dy, dt = phi[t, y, x]
        assert lv.dtilde[t + dt, y + dy, x + dx] == 1
        # the stored value is the FP64 definition for the kept shift
        assert d2[t, y, x] == O.dist(lv.x, (x, y, t), (x + dx, y + dy, t + dt), fp64=True)


def test_fp64_and_fp32_searches_differ_only_at_near_ties():
    lv, phi0 = _level()
    p32, p64 = phi0.copy(), phi0.copy()
    d32 = np.full(lv.hole.shape, np.inf, np.float32)
    d64 = np.full(lv.hole.shape, np.inf, np.float64)
    O.ann(lv.x, lv.htilde, lv.dtilde, p32, d32, n_pm=10, key=(5, 0), sub_sweeps=2)
    O.ann(lv.x, lv.htilde, lv.dtilde, p64, d64, n_pm=10, key=(5, 0), sub_sweeps=2)
    t = lv.htilde == 1
    same = (p32 == p64).all(axis=-1) & t
    # almost every decision is the same
    assert same.sum() >= 0.98 * t.sum()
    # where they agree, the FP32 distance is the FP64 one to FP32 accuracy
    rel = np.abs(d32[same].astype(np.float64) - d64[same]) / np.maximum(d64[same], 1e-30)
    assert rel.max() <= 2e-5
    # where they differ, the two searches ended at shifts whose FP64
    # distances are within the same accuracy of each other, or the searches
    # went separate ways after a near-tie: either way no FP32 decision is far
    # from the FP64 one
    assert np.median(rel) <= 1e-6
