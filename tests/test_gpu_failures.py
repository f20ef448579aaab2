"""Failures made on the host, without faulting the GPU (vi_config.mem_limit
refuses allocations beyond a per-context budget as a full device would): a
run within vi_footprint_bytes succeeds with the unlimited result, so the
admission bound holds; a run below it fails with VI_ERR_OOM and a message,
and the context is destroyed cleanly; a batch refuses the clip and goes on
with the others; the server reports the failed request and serves the next."""
import ctypes

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


def _footprint(c, **cfg):
    T, H, W = c.mask.shape
    conf = vi.default_config(**cfg)
    return int(vi.load().vi_footprint_bytes(ctypes.byref(conf), W, H, T, int(c.mask.sum())))


def _run(c, **cfg):
    with vi.Context(**cfg) as ctx:
        ctx.upload(c.rgb, c.mask)
        ctx.run()
        return ctx.fetch_result()


@pytest.mark.parametrize("storage", [0, 1])
def test_footprint_is_enough_and_less_is_refused(storage):
    c = synth.layered_clip(96, 64, 16, 2, (10, 20), 0.08, 3, 2001)
    cfg = dict(levels=3, seed=8, storage=storage)
    want = _run(c, **cfg)
    fp = _footprint(c, **cfg)
    got = _run(c, mem_limit=fp, **cfg)
    assert (got.view(np.uint32) == want.view(np.uint32)).all()
    with pytest.raises(vi.ViError, match="OOM"):
        _run(c, mem_limit=fp // 4, **cfg)
    # the device is unharmed: the next context runs as before
    assert (_run(c, **cfg).view(np.uint32) == want.view(np.uint32)).all()


def test_batch_refuses_the_clip_and_goes_on():
    a = synth.small_layered(W=64, H=48, T=10, levels=2, seed=2002)
    b = synth.small_layered(W=72, H=56, T=12, levels=2, seed=2003)
    with vi.Batch(levels=2) as bt:
        ia = bt.add(a.rgb, a.mask, seed=1, clip=0)
        with pytest.raises(vi.ViError):
            bt.add(b.rgb, b.mask, seed=2, clip=1, mem_limit=1 << 20)
        bt.run()
        want = _run(a, levels=2, seed=1, clip=0)
        assert (bt.fetch(ia).view(np.uint32) == want.view(np.uint32)).all()


def test_server_reports_the_failed_request():
    a = synth.small_layered(W=64, H=48, T=10, levels=2, seed=2004)
    with vi.Server(1 << 30, 2, levels=2) as srv:
        bad = srv.submit(a.rgb, a.mask, seed=3, mem_limit=1 << 20)
        good = srv.submit(a.rgb, a.mask, seed=3)
        assert srv.wait(bad, 60.0) == -1
        with pytest.raises(vi.ViError, match="memory limit"):
            srv.release(bad)
        assert srv.wait(good, 60.0) == 1
        assert (srv.release(good).view(np.uint32) == _run(a, levels=2, seed=3).view(np.uint32)).all()
