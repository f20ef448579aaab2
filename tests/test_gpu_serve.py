"""The server over both CUDA backends (the shared batch, and one
priority stream per request): requests that arrive while others run, under
a memory budget that holds only some of them at once, each come back
bit-identical to the same clip run alone with vi_run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1503_05528_gb300 import synth, vi  # noqa: E402
from paper_1503_05528_gb300.serve import CudaBackend, Server, StreamBackend  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


SIZES = [(96, 64, 12, 0.06), (72, 56, 16, 0.08), (128, 80, 10, 0.05), (64, 48, 20, 0.10),
         (80, 72, 14, 0.07)]


def _alone(clip, seed, tag):
    with vi.Context(levels=0, use_texture=1, seed=seed, clip=tag) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.run()
        return ctx.fetch_result()


@pytest.mark.parametrize("kind", ["batch", "streams"])
def test_served_equals_alone(kind):
    clips = [synth.fast_layered_clip(W, H, T, f, seed=2100 + i) for i, (W, H, T, f) in enumerate(SIZES)]
    if kind == "batch":
        backend = CudaBackend(levels=0, use_texture=1)
    else:
        backend = StreamBackend(max_workers=4, device=0, levels=0, use_texture=1)
    try:
        probe = Server(backend, 1 << 62)
        fps = []
        for c in clips:
            probe.submit(c.rgb, c.mask)
            fps.append(probe.queue[-1].footprint)
        probe.queue.clear()
        assert all(f > 0 for f in fps)
        # room for the two largest at once: later requests wait for memory
        budget = sum(sorted(fps)[-2:])
        srv = Server(backend, budget, max_slots=8)
        tickets = [srv.submit(clips[0].rgb, clips[0].mask, seed=50, clip=0),
                   srv.submit(clips[1].rgb, clips[1].mask, seed=51, clip=1)]
        srv.step()
        for i in range(2, len(clips)):                 # arrive while others iterate
            tickets.append(srv.submit(clips[i].rgb, clips[i].mask, seed=50 + i, clip=i))
            srv.step()
            assert srv.used <= budget
        while srv.step():
            assert srv.used <= budget
        assert srv.used == 0 and len(srv.done) == len(clips)
        assert srv.max_concurrent >= 2
        for i, t in enumerate(tickets):
            got = srv.done[t].result
            want = _alone(clips[i], 50 + i, i)
            assert (got.view(np.uint32) == want.view(np.uint32)).all(), i
    finally:
        backend.close()
