"""The temporal subsampling option (vi_config.time_subsample; Sec. 3.6 uses it
once, for long occlusions) against the oracle: per-level sizes, set codes
bit-exact and channels within tolerance; the level transition (shifts
upsampled with dt doubled, coarse parent at t/2) bit-exact in the shift map
and distances; a whole run and a batch."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1503_05528_gb300 import synth, vi  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_COLOUR = 1e-4
TOL_TEXTURE = 1e-4 * math.sqrt(50.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


def _make(seed, levels=2, T=14):
    clip = synth.small_layered(W=72, H=56, T=T, levels=levels, seed=seed)
    pyr = O.build_pyramid(clip.rgb, clip.mask, levels, True, tsub=True)
    ctx = vi.Context(levels=levels, use_texture=1, seed=seed, time_subsample=1)
    ctx.upload(clip.rgb, clip.mask)
    ctx.build_pyramid()
    return clip, pyr, ctx


@pytest.mark.parametrize("T,levels", [(20, 3), (11, 2)])
def test_sets_and_pyramid(T, levels):
    # the coarsest level needs at least 5 frames for a whole 5x5x5 source patch
    clip, pyr, ctx = _make(1540, levels=levels, T=T)
    with ctx:
        for level, lv in enumerate(pyr):
            info = ctx.level_info(level)
            assert (info["T"], info["H"], info["W"]) == lv.hole.shape
            code = ctx.get_masks(level)
            assert (lv.hole == (code & 1)).all()
            assert (lv.htilde == ((code >> 1) & 1)).all()
            assert (lv.dtilde == ((code >> 2) & 1)).all()
            gx = ctx.get_channels(level)
            assert np.abs(gx[..., :3] - lv.x[..., :3]).max() <= 2e-6
            assert np.abs(gx[..., 3:] - lv.x[..., 3:]).max() <= 1e-5 * math.sqrt(50.0)


def test_level_transition():
    clip, pyr, ctx = _make(1541, levels=2)
    with ctx:
        coarse, fine = pyr[1], pyr[0]
        rng = np.random.default_rng(5)
        xc = coarse.x.copy()
        h = coarse.hole.astype(bool)
        xc[h] = rng.random((int(h.sum()), xc.shape[-1]), dtype=np.float32) * np.float32(0.8) + np.float32(0.1)
        phic = O.init_nnf(coarse.htilde, coarse.dtilde, (47, 0), O.tag(O.PURPOSE_INIT, 1))
        d2c = np.full(coarse.hole.shape, np.inf, np.float32)
        O.ann(xc, coarse.htilde, coarse.dtilde, phic, d2c, n_pm=3, key=(47, 0))
        xf = fine.x.copy()
        ctx.set_channels(1, xc)
        ctx.set_nnf(1, phic, d2c)
        ctx.set_channels(0, xf)
        ctx.next_level(1)
        gphi, gd2 = ctx.get_nnf(0)
        gx = ctx.get_channels(0)
        coarse.x, coarse.phi, coarse.d2 = xc, phic, d2c
        fine.x = xf.copy()
        O.next_level(coarse, fine, O.Params(seed=1541, time_subsample=True), 0)
        m = fine.htilde == 1
        assert (gphi[m] == fine.phi[m]).all()
        assert (gd2[m].view(np.uint32) == fine.d2[m].view(np.uint32)).all()
        assert np.abs(gx[..., :3] - fine.x[..., :3]).max() <= TOL_COLOUR
        assert np.abs(gx[..., 3:] - fine.x[..., 3:]).max() <= TOL_TEXTURE


def test_full_run_and_batch():
    clips = [synth.small_layered(W=64, H=48, T=T, levels=2, seed=1550 + T) for T in (12, 9)]
    outs = []
    for i, c in enumerate(clips):
        with vi.Context(levels=2, seed=60 + i, clip=i, time_subsample=1) as ctx:
            ctx.upload(c.rgb, c.mask)
            ctx.run()
            out = ctx.fetch_result()
        assert np.isfinite(out).all()
        assert np.array_equal(out[c.mask == 0], c.rgb[c.mask == 0])
        outs.append(out)
    with vi.Batch(levels=2, time_subsample=1) as b:
        ids = [b.add(c.rgb, c.mask, seed=60 + i, clip=i) for i, c in enumerate(clips)]
        b.run()
        for cid, want in zip(ids, outs):
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all()
