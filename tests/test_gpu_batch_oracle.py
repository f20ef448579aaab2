"""Parity of a batch round (vi_batch_step: the persistent batch kernels
k_rescore_batch, k_ann_step_batch[_warp] and k_vote_batch over several clips
at once) with the oracle's search and vote, on injected state.

Three clips of different sizes and level counts share every launch. Before
each round, every clip gets an oracle state at its current level (channels
with the occluded voxels filled by seeded values, a shift map from the
oracle's initialisation); the round runs; then each clip's shift map and
distances must equal the oracle's Jacobi search (Algorithm 1, rescore + n_pm
sweeps, the clip's own Philox key, tag and counter word) bit for bit, and its
voxels the oracle's vote (Eq. 4/5, Eq. 9) within 1e-4. Warps of the
warp-shared kernel hold targets of two clips at the list boundaries."""
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


def _clips():
    return [synth.small_layered(W=72, H=56, T=14, levels=2, seed=1514),
            synth.small_layered(W=37, H=29, T=9, levels=1, seed=1515),
            synth.small_layered(W=48, H=40, T=10, levels=2, seed=1516)]


def _state(lv, seed, level, rnd):
    rng = np.random.default_rng(1000 * rnd + seed)
    x = lv.x.copy()
    h = lv.hole.astype(bool)
    x[h] = rng.random((int(h.sum()), x.shape[-1]), dtype=np.float32) * np.float32(0.8) + np.float32(0.1)
    phi = O.init_nnf(lv.htilde, lv.dtilde, (seed + rnd, 0), O.tag(O.PURPOSE_INIT, level))
    d2 = np.full(lv.hole.shape, np.inf, np.float32)
    return x, phi, d2


@pytest.mark.parametrize("lanes,storage,sub_sweeps", [(0, 0, 1), (1, 0, 1), (32, 0, 1), (0, 2, 1), (32, 2, 1),
                                                      (0, 0, 2), (32, 0, 2), (32, 2, 2), (32, 1, 2), (1, 0, 3)])
def test_batch_rounds_match_oracle_search_and_vote(lanes, storage, sub_sweeps):
    clips = _clips()
    pyrs = [O.build_pyramid(c.rgb, c.mask, c.levels, True) for c in clips]
    seeds = [301, 302, 303]
    compared = 0
    with vi.Batch(levels=0, lanes_per_target=lanes, storage=storage, sub_sweeps=sub_sweeps) as b:
        ids = [b.add(c.rgb, c.mask, levels=c.levels, seed=s, clip=i, max_outer=3, stop=0.0)
               for i, (c, s) in enumerate(zip(clips, seeds))]
        for rnd in range(12):
            plan = {}
            for i, cid in enumerate(ids):
                done, level = b.poll(cid)
                if done:
                    continue
                ctx, call = b.clip_context(cid)
                lv = pyrs[i][level]
                x, phi, d2 = _state(lv, seeds[i], level, rnd)
                ctx.set_channels(level, x)
                ctx.set_nnf(level, phi, d2)
                plan[i] = (level, call, x, phi, d2)
            if not plan:
                break
            b.step()
            for i, (level, call, x, phi, d2) in plan.items():
                done, now = b.poll(ids[i])
                if done or now != level:
                    continue      # moved on: its level state was rewritten
                lv = pyrs[i][level]
                ophi, od2 = phi.copy(), d2.copy()
                O.ann(x, lv.htilde, lv.dtilde, ophi, od2, n_pm=10, schedule="JAC", key=(seeds[i], 0),
                      tag_base=O.tag(O.PURPOSE_SEARCH, level, call), clip=i, sub_sweeps=sub_sweeps)
                ox, _ = O.vote(x, lv.hole, lv.htilde, ophi, od2, weighted=True, n_diff=3)
                ctx, _ = b.clip_context(ids[i])
                gphi, gd2 = ctx.get_nnf(level)
                gx = ctx.get_channels(level)
                m = lv.htilde == 1
                assert (gphi[m] == ophi[m]).all(), f"clip {i} level {level} call {call}: shifts"
                assert (gd2[m].view(np.uint32) == od2[m].view(np.uint32)).all(), \
                    f"clip {i} level {level} call {call}: distances"
                assert np.abs(gx[..., :3] - ox[..., :3]).max() <= TOL_COLOUR
                assert np.abs(gx[..., 3:] - ox[..., 3:]).max() <= TOL_TEXTURE
                compared += 1
    # two compared rounds per level of every clip (the third moves the clip on)
    assert compared == 2 * sum(c.levels for c in clips)
