"""Full-size runs of the CUDA path, in the configuration bench.py times (one
vi_run of the whole method), checked on sampled outputs the oracle computes
one by one from the same input (sets and texture features on small crops
around the samples) and on properties that hold at any size:

- every target's shift lands in D~;
- the stored distance of a shift is the distance recomputed from the stored
  channels (numpy, FP64, within the FP32 rounding);
- known voxels come back exactly as given, and every occluded voxel is a copy
  of a known voxel p + phi(q) for some q in its patch (Eq. 6);
- each coarse occlusion voxel is the OR of its fine children.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1503_05528_gb300 import vi  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


def _numpy_d2(x, p, s):
    """Eq. 2 / 7b in FP64 for an interior source, clipped target patch."""
    T, H, W, _ = x.shape
    acc = 0.0
    for dt in range(-2, 3):
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                r = (p[2] + dt, p[1] + dy, p[0] + dx)
                if not (0 <= r[0] < T and 0 <= r[1] < H and 0 <= r[2] < W):
                    continue
                q = (s[2] + dt, s[1] + dy, s[0] + dx)
                df = x[r].astype(np.float64) - x[q].astype(np.float64)
                acc += float((df * df).sum())
    return acc / 125.0


def _crop(a, t, y, x, r, rt):
    T, H, W = a.shape[:3]
    t0, t1 = max(t - rt, 0), min(t + rt + 1, T)
    y0, y1 = max(y - r, 0), min(y + r + 1, H)
    x0, x1 = max(x - r, 0), min(x + r + 1, W)
    return a[t0:t1, y0:y1, x0:x1], (t - t0, y - y0, x - x0), (t0 == 0 or t1 == T, y0 == 0 or y1 == H,
                                                               x0 == 0 or x1 == W)


def _check_run(workload, n_samples, seed):
    clip = bench.make_clip(0, workload)
    rng = np.random.default_rng(seed)
    with vi.Context(levels=clip.levels, use_texture=1, seed=1503) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.build_pyramid()
        code0 = ctx.get_masks(0)
        x0 = ctx.get_channels(0)
        codes = [ctx.get_masks(l) for l in range(clip.levels)]
        ctx.upload(clip.rgb, clip.mask)
        ctx.run()
        out = ctx.fetch_result()
        ctx.rescore(0)
        x = ctx.get_channels(0)
        phi, d2 = ctx.get_nnf(0)
        stats = ctx.stats()
    T, H, W = clip.mask.shape
    assert all(1 <= n <= 20 for n in stats["outer"][:clip.levels])

    # sets D~ / H~ at sampled voxels against the oracle on a crop (radius 4:
    # the crop's own border is at least 2 voxels from the sample unless it
    # is the video's border)
    for _ in range(n_samples):
        t, y, xx = int(rng.integers(0, T)), int(rng.integers(0, H)), int(rng.integers(0, W))
        m, (ct, cy, cx), _ = _crop(clip.mask, t, y, xx, 4, 4)
        ht, dt_ = O.masks(np.ascontiguousarray(m))
        c = code0[t, y, xx]
        assert ht[ct, cy, cx] == (c >> 1) & 1
        assert dt_[ct, cy, cx] == (c >> 2) & 1
        assert (c & 1) == clip.mask[t, y, xx]

    # texture features (Eq. 7, window 2^(L-1), one frame) at sampled known
    # voxels against the oracle on a crop of radius side/2 + 2
    side = 2 ** (clip.levels - 1)
    s_lam = O.sqrt_lambda(50.0)
    checked = 0
    while checked < n_samples:
        t, y, xx = int(rng.integers(0, T)), int(rng.integers(0, H)), int(rng.integers(0, W))
        if clip.mask[t, y, xx]:
            continue
        r = side // 2 + 2
        cy0, cy1, cx0, cx1 = max(y - r, 0), min(y + r + 1, H), max(xx - r, 0), min(xx + r + 1, W)
        # a crop whose edge is not the frame edge changes one-sided differences
        # only at that edge, which is outside the window of the centre sample
        rgb = np.ascontiguousarray(clip.rgb[t:t + 1, cy0:cy1, cx0:cx1])
        hm = np.ascontiguousarray(clip.mask[t:t + 1, cy0:cy1, cx0:cx1])
        Tf = O.texture_features(rgb, hm, side)
        want = (s_lam * Tf[0, y - cy0, xx - cx0]).astype(np.float32)
        assert np.abs(x0[t, y, xx, 3:5] - want).max() <= 2e-5 * math.sqrt(50.0)
        checked += 1

    # shift validity and distances of stored shifts (all level-0 targets)
    tt, yy, xs = np.nonzero((code0 >> 1) & 1)
    st, sy, sx = tt + phi[tt, yy, xs, 2], yy + phi[tt, yy, xs, 1], xs + phi[tt, yy, xs, 0]
    inb = (st >= 0) & (st < T) & (sy >= 0) & (sy < H) & (sx >= 0) & (sx < W)
    assert inb.all()
    assert ((code0[st, sy, sx] >> 2) & 1).all()
    for i in rng.choice(len(tt), n_samples, replace=False):
        p = (int(xs[i]), int(yy[i]), int(tt[i]))
        s = (int(sx[i]), int(sy[i]), int(st[i]))
        want = _numpy_d2(x, p, s)
        assert d2[p[2], p[1], p[0]] == pytest.approx(want, rel=2e-5, abs=1e-9)

    # outputs: known voxels unchanged; occluded voxels copy a contributor
    known = clip.mask == 0
    assert (out[known] == clip.rgb[known]).all()
    ht_, hy, hx = np.nonzero(clip.mask)
    for i in rng.choice(len(ht_), n_samples, replace=False):
        t, y, xx = int(ht_[i]), int(hy[i]), int(hx[i])
        cands = []
        for a in range(-2, 3):
            for b in range(-2, 3):
                for c in range(-2, 3):
                    q = (t + a, y + b, xx + c)
                    if 0 <= q[0] < T and 0 <= q[1] < H and 0 <= q[2] < W:
                        f = phi[q]
                        cands.append(clip.rgb[t + f[2], y + f[1], xx + f[0]])
        assert any((out[t, y, xx] == v).all() for v in cands)

    # occlusion pyramid: OR of children
    for l in range(1, clip.levels):
        fine = codes[l - 1] & 1
        coarse = codes[l] & 1
        Tl, Hl, Wl = coarse.shape
        pad = np.zeros((fine.shape[0], 2 * Hl, 2 * Wl), np.uint8)
        pad[:, :fine.shape[1], :fine.shape[2]] = fine
        orr = pad.reshape(Tl, Hl, 2, Wl, 2).max(axis=(2, 4))
        assert (orr == coarse).all()


def test_bench_workload_full_size():
    _check_run("layered_320x240x60", 200, 1)


def test_hd_workload_full_size():
    _check_run("layered_1280x720x100", 120, 2)


def _golden_seq_energy():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "seq_energy_layered_320x240x60.txt")
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = [float(x) for x in v]
    return vals


def test_full_run_energy_vs_the_sequential_oracle():
    # the whole method in the library's default configuration on the
    # 320x240x60 workload (parallel Jacobi sweeps) against the oracle's
    # sequential sweep (Algorithm 1 as printed), compared by the Eq. 1 energy
    # over H and over H~ at level 0 after the last iteration and before the
    # final step, both evaluated by the oracle (the stored value was written
    # by tests/golden/make_seq_energy.py): within 2%. A Jacobi sweep spreads a
    # good shift one voxel; the default's two propagation sweeps per
    # iteration bring the energy within 2% of the sequential sweep's.
    gold = _golden_seq_energy()
    bound = 1.02
    clip = bench.make_clip(0, "layered_320x240x60")
    sub_sweeps = vi.default_config().sub_sweeps
    with vi.Context(levels=clip.levels, use_texture=1, seed=1503) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.prepare()
        for level in range(clip.levels - 1, -1, -1):
            ctx.iterate(level)
            if level > 0:
                ctx.next_level(level)
        x = ctx.get_channels(0)
        phi, _ = ctx.get_nnf(0)
        code = ctx.get_masks(0)
    e_h, e_ht = O.energy(x, code & 1, (code >> 1) & 1, phi)
    print(f"sub_sweeps {sub_sweeps}: E_H {e_h:.4f} (sequential {gold['E_H'][0]:.4f}), "
          f"E_H~ {e_ht:.4f} ({gold['E_Htilde'][0]:.4f})")
    assert e_h <= bound * gold["E_H"][0], (e_h, gold["E_H"][0])
    assert e_ht <= bound * gold["E_Htilde"][0], (e_ht, gold["E_Htilde"][0])
