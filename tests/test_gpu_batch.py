"""Batches of uneven clips (vi_batch_*): every clip's inpainted video, shift
map and iteration counts are bit-identical to the same clip run alone with
vi_run, whether the batch is filled up front or clips join and leave while
others are iterating (continuous batching)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1503_05528_gb300 import synth, vi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


# uneven clips: (W, H, T, levels, hole fraction, seed)
SPECS = [(72, 56, 14, 2, 0.08, 1601), (96, 64, 10, 2, 0.05, 1602), (48, 40, 12, 1, 0.10, 1603),
         (120, 80, 16, 3, 0.06, 1604), (64, 64, 8, 1, 0.08, 1605), (88, 48, 20, 2, 0.12, 1606)]


def _clip(spec):
    W, H, T, L, frac, seed = spec
    return synth.layered_clip(W, H, T, 2, (10, 20), frac, L, seed, name=f"c{seed}")


def _alone(clip, seed, tag, with_evals=False):
    with vi.Context(levels=clip.levels, seed=seed, clip=tag) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.run()
        out = ctx.fetch_result()
        phi, _ = ctx.get_nnf(0)
        st = ctx.stats()
    if with_evals:
        return out, phi, st["outer"][:clip.levels], st["evals"]
    return out, phi, st["outer"][:clip.levels]


@pytest.mark.parametrize("lanes", [0, 32])
def test_batch_equals_alone(lanes):
    # lanes 32: the warp-shared step, whose warps straddle clip boundaries
    clips = [_clip(s) for s in SPECS]
    with vi.Batch(lanes_per_target=lanes) as b:
        ids = [b.add(c.rgb, c.mask, levels=c.levels, seed=100 + i, clip=i) for i, c in enumerate(clips)]
        b.run()
        alone_evals = 0
        for i, (cid, c) in enumerate(zip(ids, clips)):
            assert b.poll(cid) == (1, 0)
            got = b.fetch(cid)
            want, _, outer, ev = _alone(c, 100 + i, i, with_evals=True)
            alone_evals += ev
            assert (got.view(np.uint32) == want.view(np.uint32)).all(), i
            assert b.clip_stats(cid)["outer"][:c.levels] == outer
        s = b.stats()
        assert s["rounds"] >= 1 and s["evals"] > 0
        # the batch makes exactly the evaluations the clips make alone
        assert s["evals"] == alone_evals


def test_continuous_batching_join_and_leave():
    clips = [_clip(s) for s in SPECS[:4]]
    with vi.Batch() as b:
        first = [b.add(c.rgb, c.mask, levels=c.levels, seed=200 + i, clip=i) for i, c in enumerate(clips[:2])]
        b.step()
        b.step()
        late = b.add(clips[2].rgb, clips[2].mask, levels=clips[2].levels, seed=202, clip=2)
        gone = b.add(clips[3].rgb, clips[3].mask, levels=clips[3].levels, seed=203, clip=3)
        b.step()
        b.remove(gone)                       # leaves while iterating
        n = 1
        while n:
            n = b.step()
        for i, cid in enumerate(first + [late]):
            want, _, _ = _alone(clips[i], 200 + i, i)
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), i
        with pytest.raises(vi.ViError):
            b.poll(gone)


def test_batch_rejects_mismatched_channels():
    with vi.Batch(use_texture=1) as b:
        c = _clip(SPECS[2])
        with pytest.raises(vi.ViError):
            b.add(c.rgb, c.mask, use_texture=0)


def test_batch_multi_radius_search_equals_alone():
    clips = [_clip(s) for s in SPECS[:3]]
    with vi.Batch(rs_mode=1) as b:
        ids = [b.add(c.rgb, c.mask, levels=c.levels, seed=300 + i, clip=i) for i, c in enumerate(clips)]
        b.run()
        for i, (cid, c) in enumerate(zip(ids, clips)):
            with vi.Context(levels=c.levels, seed=300 + i, clip=i, rs_mode=1) as ctx:
                ctx.upload(c.rgb, c.mask)
                ctx.run()
                want = ctx.fetch_result()
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), i
        with pytest.raises(vi.ViError):   # a batch's clips share its propagation sweeps per iteration
            b.add(clips[0].rgb, clips[0].mask, sub_sweeps=3)


def test_warp_shared_batch_mixed_search_modes():
    # clips with Eq. 3 and with the multi-radius search (different numbers of
    # random candidates, different r_max) share warps of the warp-shared step
    clips = [_clip(s) for s in SPECS[:5]]
    modes = [1, 0, 1, 0, 1]
    with vi.Batch(lanes_per_target=32) as b:
        ids = [b.add(c.rgb, c.mask, levels=c.levels, seed=400 + i, clip=i, rs_mode=m)
               for i, (c, m) in enumerate(zip(clips, modes))]
        b.run()
        for i, (cid, c, m) in enumerate(zip(ids, clips, modes)):
            with vi.Context(levels=c.levels, seed=400 + i, clip=i, rs_mode=m) as ctx:
                ctx.upload(c.rgb, c.mask)
                ctx.run()
                want = ctx.fetch_result()
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), i


@pytest.mark.parametrize("lanes", [0, 32])
def test_batch_with_sub_sweeps_is_identical_to_vi_run(lanes):
    # two propagation sweeps per iteration: a clip's batch result equals the
    # single-clip run with the same setting, bit for bit
    clips = [_clip(s) for s in SPECS[:4]]
    with vi.Batch(sub_sweeps=2, lanes_per_target=lanes) as b:
        ids = [b.add(c.rgb, c.mask, levels=c.levels, seed=500 + i, clip=i) for i, c in enumerate(clips)]
        b.run()
        for i, (cid, c) in enumerate(zip(ids, clips)):
            with vi.Context(levels=c.levels, seed=500 + i, clip=i, sub_sweeps=2, lanes_per_target=lanes) as ctx:
                ctx.upload(c.rgb, c.mask)
                ctx.run()
                want = ctx.fetch_result()
                outer = ctx.stats()["outer"]
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), i
            assert b.clip_stats(cid)["outer"] == outer


@pytest.mark.parametrize("device", [False, True])
def test_add_many_prepares_concurrently_with_the_same_results(device):
    # vi_batch_add_many uploads and prepares the clips on streams of their own
    # from several threads; every clip's result and iteration counts are the
    # ones it gets alone through vi_run, bit for bit
    clips = [_clip(s) for s in SPECS[:5]]
    items = []
    for i, c in enumerate(clips):
        rgb, mask = (torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()) if device else (c.rgb, c.mask)
        items.append((rgb, mask, dict(levels=c.levels, seed=600 + i, clip=i)))
    stream = torch.cuda.current_stream()
    with vi.Batch(stream=stream.cuda_stream, lanes_per_target=32) as b:
        ids = b.add_many(items, n_threads=3)
        assert sorted(ids) == list(range(5))
        b.run()
        for i, (cid, c) in enumerate(zip(ids, clips)):
            with vi.Context(levels=c.levels, seed=600 + i, clip=i) as ctx:
                ctx.upload(c.rgb, c.mask)
                ctx.run()
                want = ctx.fetch_result()
                outer = ctx.stats()["outer"]
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), i
            assert b.clip_stats(cid)["outer"] == outer


def test_add_many_reports_a_failing_clip_and_adds_the_others():
    clips = [_clip(s) for s in SPECS[:3]]
    bad = synth.Clip("all occluded", clips[0].rgb.copy(), np.ones_like(clips[0].mask), clips[0].levels, True)
    items = [(c.rgb, c.mask, dict(levels=c.levels, seed=700 + i, clip=i)) for i, c in enumerate(clips)]
    items.insert(1, (bad.rgb, bad.mask, dict(levels=bad.levels, seed=799, clip=9)))
    with vi.Batch() as b:
        with pytest.raises(vi.ViError) as e:
            b.add_many(items)
        ids = e.value.ids
        assert ids[1] == -1 and all(x >= 0 for k, x in enumerate(ids) if k != 1)
        assert e.value.statuses[1] != 0
        b.run()
        for k, (cid, (rgb, mask, job)) in enumerate(zip(ids, items)):
            if k == 1:
                continue
            with vi.Context(**job) as ctx:
                ctx.upload(rgb, mask)
                ctx.run()
                want = ctx.fetch_result()
            assert (b.fetch(cid).view(np.uint32) == want.view(np.uint32)).all(), k
