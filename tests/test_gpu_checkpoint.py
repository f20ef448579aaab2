"""Checkpoint and resume (vi_save_state / vi_load_state / vi_resume): a run
stopped between two iterations of any level, saved, and resumed in a fresh
context that built the same pyramid gives vi_run's output bit for bit, with
the same iteration counts; FP16 storage rebuilds its copies on load; a state
of another level, size or configuration is refused."""
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


def _whole(c, **cfg):
    with vi.Context(**cfg) as a:
        a.upload(c.rgb, c.mask)
        a.run()
        return a.fetch_result(), a.stats()["outer"]


def _stop_and_save(c, level, k0, **cfg):
    L = cfg["levels"]
    with vi.Context(**cfg) as b:
        b.upload(c.rgb, c.mask)
        b.prepare()
        for l in range(L - 1, level, -1):
            b.iterate(l)
            b.next_level(l)
        n, _ = b.iterate(level, n_outer=k0)
        assert n == k0
        return b.save_state(level)


def _resume(c, level, k0, state, **cfg):
    with vi.Context(**cfg) as r:
        r.upload(c.rgb, c.mask)
        r.build_pyramid()
        r.load_state(level, state)
        r.resume(level, k0)
        return r.fetch_result(), r.stats()["outer"]


@pytest.mark.parametrize("storage", [0, 2])
def test_resume_at_every_level(storage):
    c = synth.layered_clip(96, 64, 16, 2, (10, 20), 0.08, 3, 1901)
    cfg = dict(levels=3, seed=77, clip=2, storage=storage)
    want, outer = _whole(c, **cfg)
    for level in range(3):
        assert outer[level] >= 2          # the whole run went on past the first iteration
        state = _stop_and_save(c, level, 1, **cfg)
        got, outer_r = _resume(c, level, 1, state, **cfg)
        assert (got.view(np.uint32) == want.view(np.uint32)).all(), level
        assert outer_r[level] == outer[level] - 1
        assert outer_r[:level] == outer[:level]


def test_state_checks():
    c = synth.small_layered(W=64, H=48, T=12, levels=2, seed=1902)
    with vi.Context(levels=2, seed=3) as a:
        a.upload(c.rgb, c.mask)
        a.prepare()
        a.iterate(1, n_outer=1)
        s1 = a.save_state(1)
        s0 = a.save_state(0)
        with pytest.raises(vi.ViError):
            a.load_state(0, s1)                      # another level's state
        with pytest.raises(vi.ViError):
            a.load_state(1, s1[:-4])                 # truncated
        bad = bytearray(s1)
        bad[0] ^= 1
        with pytest.raises(vi.ViError):
            a.load_state(1, bytes(bad))              # not a state
        a.load_state(1, s1)
        a.load_state(0, s0)
    with vi.Context(levels=2, seed=3, use_texture=0) as b:
        b.upload(c.rgb, c.mask)
        b.build_pyramid()
        with pytest.raises(vi.ViError):
            b.load_state(1, s1)                      # five channels into a three-channel context
