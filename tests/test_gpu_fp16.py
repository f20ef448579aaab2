"""FP16 storage (vi_config.storage = 2: screening at every level; storage 1
screens only levels larger than the L2 cache, so these small clips run it as
FP32). The PatchMatch step screens the random-search candidates on FP16
copies of the channels under a rigorous error bound and takes its decision
on the FP32 distance, so shift maps, distances and evaluation counts equal
the oracle's bit for bit, and whole runs equal the FP32-storage runs bit for
bit. The screening must reject most candidates (that is its point) and must
let every candidate through when the channel magnitudes leave the FP16
range."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1503_05528_gb300 import synth, vi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


CASES = {
    "tiny_rgb": dict(clip=lambda: synth.tiny_translation_clip(), levels=1, tex=False),
    "layered_tex": dict(clip=lambda: synth.small_layered(W=72, H=56, T=14, levels=2, seed=1514),
                        levels=2, tex=True),
    "odd_sizes": dict(clip=lambda: synth.small_layered(W=37, H=29, T=9, levels=1, seed=1515),
                      levels=1, tex=True),
}


def _make(case, seed, n_pm=10, lanes=0):
    spec = CASES[case]
    clip = spec["clip"]()
    pyr = O.build_pyramid(clip.rgb, clip.mask, spec["levels"], spec["tex"])
    ctx = vi.Context(levels=spec["levels"], use_texture=int(spec["tex"]), seed=seed, n_pm=n_pm, storage=2, sub_sweeps=2,
                     lanes_per_target=lanes)
    ctx.upload(clip.rgb, clip.mask)
    ctx.build_pyramid()
    return clip, pyr, ctx


def _state(lv, level, seed, scale=1.0):
    """An oracle state: the level's channels (times scale) with the occluded
    voxels filled by seeded values, and the oracle's random shift map."""
    rng = np.random.default_rng(5)
    x = lv.x.copy()
    h = lv.hole.astype(bool)
    x[h] = rng.random((int(h.sum()), x.shape[-1]), dtype=np.float32) * np.float32(0.8) + np.float32(0.1)
    x = (x * np.float32(scale)).astype(np.float32)
    phi = O.init_nnf(lv.htilde, lv.dtilde, (seed, 0), O.tag(O.PURPOSE_INIT, level))
    d2 = np.full(lv.hole.shape, np.inf, np.float32)
    return x, phi, d2


def _ann_check(ctx, lv, level, x, phi, d2, seed, n_pm, call):
    ctx.set_channels(level, x)
    ctx.set_nnf(level, phi, d2)
    s0 = ctx.stats()
    ctx.ann(level, call)
    s1 = ctx.stats()
    gphi, gd2 = ctx.get_nnf(level)
    o_evals = O.ann(x, lv.htilde, lv.dtilde, phi, d2, n_pm=n_pm, schedule="JAC", key=(seed, 0),
                    tag_base=O.tag(O.PURPOSE_SEARCH, level, call), sub_sweeps=2)
    m = lv.htilde == 1
    assert (gphi[m] == phi[m]).all()
    assert (gd2[m].view(np.uint32) == d2[m].view(np.uint32)).all()
    assert s1["evals"] - s0["evals"] == o_evals
    return {k: s1[k] - s0[k] for k in ("screened", "screen_passed", "step_gathered_h", "step_gathered")}


@pytest.mark.parametrize("lanes", [0, 32])
@pytest.mark.parametrize("case,n_pm,call", [("tiny_rgb", 10, 0), ("layered_tex", 10, 3),
                                            ("odd_sizes", 3, 17)])
def test_ann_fp16_bit_exact(case, n_pm, call, lanes):
    # lanes 32: the warp-shared form screens and gathers with lane groups of
    # the warp; the decisions are the same
    clip, pyr, ctx = _make(case, seed=31, n_pm=n_pm, lanes=lanes)
    with ctx:
        for level, lv in enumerate(pyr):
            x, phi, d2 = _state(lv, level, 31)
            c = _ann_check(ctx, lv, level, x, phi, d2, 31, n_pm, call)
            assert c["screened"] > 0 and c["step_gathered_h"] > 0
            assert c["screen_passed"] < c["screened"]


@pytest.mark.parametrize("scale", [1000.0, 1e-3])
def test_ann_fp16_scaled_values(scale):
    # the bound follows the magnitudes: large values and values near the FP16
    # subnormal range keep the decisions exact
    clip, pyr, ctx = _make("layered_tex", seed=41)
    with ctx:
        lv = pyr[0]
        x, phi, d2 = _state(lv, 0, 41, scale=scale)
        c = _ann_check(ctx, lv, 0, x, phi, d2, 41, 10, 0)
        assert c["screened"] > 0


def test_ann_fp16_out_of_range_passes_everything():
    # one value beyond the FP16 range: no candidate may be rejected on FP16
    clip, pyr, ctx = _make("layered_tex", seed=43)
    with ctx:
        lv = pyr[1]
        x, phi, d2 = _state(lv, 1, 43)
        known = np.argwhere(lv.hole == 0)
        t, y, xx = known[len(known) // 2]
        x[t, y, xx, 0] = np.float32(1.0e5)
        c = _ann_check(ctx, lv, 1, x, phi, d2, 43, 10, 0)
        assert c["screened"] > 0 and c["screen_passed"] == c["screened"]


def _run(clip, storage, seed, tag):
    with vi.Context(levels=clip.levels, use_texture=int(clip.use_texture), seed=seed, clip=tag,
                    storage=storage) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.run()
        out = ctx.fetch_result()
        phi, d2 = ctx.get_nnf(0)
        return out, phi, d2, ctx.stats()


@pytest.mark.parametrize("which", ["layered", "fast", "tiny"])
def test_run_fp16_equals_fp32(which):
    clip = {"layered": lambda: synth.small_layered(W=96, H=72, T=16, levels=2, seed=1601),
            "fast": lambda: synth.fast_layered_clip(160, 96, 20, 0.06, seed=1602),
            "tiny": lambda: synth.tiny_translation_clip()}[which]()
    a = _run(clip, 0, 77, 1)
    b = _run(clip, 2, 77, 1)      # screening at every level
    c = _run(clip, 1, 77, 1)      # screening where a level exceeds L2: none of these
    assert (a[0].view(np.uint32) == c[0].view(np.uint32)).all() and c[3]["screened"] == 0
    assert (a[0].view(np.uint32) == b[0].view(np.uint32)).all()
    assert (a[1] == b[1]).all() and (a[2].view(np.uint32) == b[2].view(np.uint32)).all()
    assert a[3]["outer"] == b[3]["outer"] and a[3]["evals"] == b[3]["evals"]
    sb = b[3]
    assert sb["screened"] > 0 and sb["screen_passed"] < sb["screened"]
    # FP32 voxels gathered shrink to what the passed candidates need
    assert sb["step_gathered"] < a[3]["step_gathered"]


def test_batch_fp16_equals_alone_fp32():
    clips = [synth.fast_layered_clip(W, H, T, f, seed=1700 + i)
             for i, (W, H, T, f) in enumerate([(96, 64, 12, 0.06), (72, 56, 16, 0.08), (128, 80, 10, 0.05)])]
    with vi.Batch(levels=0, storage=2) as b:
        ids = [b.add(c.rgb, c.mask, seed=90 + i, clip=i) for i, c in enumerate(clips)]
        b.run()
        for i, (cid, c) in enumerate(zip(ids, clips)):
            want = _run(c, 0, 90 + i, i)[0]
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), i
        s = b.stats()
        assert s["screened"] > 0 and s["screen_passed"] < s["screened"] and s["gathered_h"] > 0
        with pytest.raises(vi.ViError):
            b.add(clips[0].rgb, clips[0].mask, storage=0)
