"""The library's own server (vi_server_*): served results are bit-identical
to the same clips run alone through vi_run (host and device buffers); the
admitted footprint never exceeds the budget; a request above the budget is
refused at submission; a failing request reports its error at release; the
server shuts down with requests still queued."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1503_05528_gb300 import synth, vi  # noqa: E402
from paper_1503_05528_gb300.serve import NativeServer, poisson_arrivals, run_load  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


def _clips():
    sizes = [(64, 48, 9), (80, 56, 12), (72, 40, 10), (96, 64, 8), (64, 64, 11)]
    return [synth.small_layered(W=W, H=H, T=T, levels=2, seed=1600 + i) for i, (W, H, T) in enumerate(sizes)]


def _alone(c, **job):
    with vi.Context(levels=2, **job) as ctx:
        ctx.upload(c.rgb, c.mask)
        ctx.run()
        return ctx.fetch_result()


def _same(a, b):
    return (np.asarray(a).view(np.uint32) == np.asarray(b).view(np.uint32)).all()


@pytest.mark.parametrize("slots", [1, 3])
def test_results_match_vi_run_alone(slots):
    clips = _clips()
    want = [_alone(c, seed=80 + i, clip=i) for i, c in enumerate(clips)]
    with vi.Server(4 << 30, slots, levels=2) as srv:
        tickets = [srv.submit(c.rgb, c.mask, seed=80 + i, clip=i) for i, c in enumerate(clips)]
        for t, w in zip(tickets, want):
            assert srv.wait(t, 120.0) == 1
            assert _same(srv.release(t), w)
        assert srv.info() == dict(queued=0, running=0, bytes_in_use=0)


def test_device_buffers():
    c = _clips()[1]
    want = _alone(c, seed=5, clip=0)
    rgb, mask = torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()
    out = torch.empty_like(rgb)
    torch.cuda.synchronize()                           # inputs complete before submission
    with vi.Server(1 << 30, 2, levels=2) as srv:
        t = srv.submit(rgb, mask, out=out, seed=5, clip=0)
        assert srv.wait(t, 120.0) == 1
        srv.release(t)
    assert _same(out.cpu().numpy(), want)


def test_budget_respected_and_too_large_refused():
    clips = _clips()
    lib = vi.load()
    import ctypes
    fps = []
    for c in clips:
        T, H, W = c.mask.shape
        cfg = vi.default_config(levels=2)
        fps.append(int(lib.vi_footprint_bytes(ctypes.byref(cfg), W, H, T, 0)))
    budget = max(fps) + min(fps) // 2          # never two of the larger requests at once
    with vi.Server(budget, 4, levels=2) as srv:
        tickets = [srv.submit(c.rgb, c.mask, seed=i, clip=i) for i, c in enumerate(clips)]
        seen = 0
        while any(srv.poll(t) == 0 for t in tickets):
            info = srv.info()
            assert info["bytes_in_use"] <= budget
            seen = max(seen, info["running"])
        assert seen >= 1
        for t in tickets:
            srv.release(t)
        big = synth.small_layered(W=256, H=192, T=20, levels=2, seed=3)
        with pytest.raises(vi.ViError, match="TOO_LARGE"):
            srv.submit(big.rgb, big.mask)


def test_failed_request_reports_and_bad_ticket():
    c = _clips()[0]
    with vi.Server(1 << 30, 2, levels=2) as srv:
        t = srv.submit(c.rgb, c.mask, sub_sweeps=17)   # rejected by the configuration check
        assert srv.wait(t, 60.0) == -1
        with pytest.raises(vi.ViError):
            srv.release(t)
        with pytest.raises(vi.ViError):
            srv.poll(t)                                # forgotten after release
        ok = srv.submit(c.rgb, c.mask, seed=1, clip=0)
        assert srv.wait(ok, 120.0) == 1
        assert _same(srv.release(ok), _alone(c, seed=1, clip=0))


def test_destroy_with_queued_requests():
    clips = _clips()
    srv = vi.Server(1 << 30, 1, levels=2)
    tickets = [srv.submit(c.rgb, c.mask, seed=i, clip=i) for i, c in enumerate(clips * 3)]
    srv.close()                                         # running one finishes, the rest fail
    assert len(tickets) == 15


def test_poisson_load_through_the_native_front():
    clips = _clips()
    reqs = [(c.rgb, c.mask, {"seed": 900 + i, "clip": i}) for i, c in enumerate(clips)]
    arrivals = poisson_arrivals(len(reqs), 50.0, seed=4)
    srv = NativeServer(2 << 30, 3, levels=2)
    wall, srv = run_load(srv, reqs, arrivals)
    srv.close()
    assert wall > 0 and len(srv.done) == len(reqs)
    for t, (rgb, mask, job) in enumerate(reqs):
        r = srv.done[t]
        assert not r.info.get("failed") and r.latency > 0
        assert _same(r.result, _alone(clips[t], **job))
