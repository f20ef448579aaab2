"""Host buffers through the C ABI: uploads from and results into pinned
(registered) host memory go through kernels reading and writing it by its
device address; pageable memory goes through the copy engine. Every form must
give the device-buffer run's output bit for bit: aligned pinned buffers (16-byte
copies), pinned views one element into their allocation (interior pointers,
single-byte copies), and pageable numpy arrays, for one clip (vi_upload /
vi_fetch_result) and for a batch (vi_batch_add_many / vi_batch_fetch)."""
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


def _pinned(a, offset):
    """A pinned host copy of numpy array a, starting `offset` elements into
    its pinned allocation (a numpy view)."""
    flat = torch.empty(a.size + offset, dtype=torch.from_numpy(np.empty(0, a.dtype)).dtype, pin_memory=True)
    assert flat.is_pinned()
    v = flat.numpy()[offset:].reshape(a.shape)
    v[...] = a
    return v


def _clips():
    return [synth.layered_clip(72, 56, 14, 2, (10, 20), 0.08, 2, 1701, name="h0"),
            synth.layered_clip(61, 47, 9, 1, (8, 14), 0.10, 1, 1702, name="h1")]


def _device_run(c, seed):
    with vi.Context(levels=c.levels, seed=seed) as ctx:
        ctx.upload(torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda())
        ctx.run()
        out = torch.empty(c.rgb.shape, dtype=torch.float32, device="cuda")
        ctx.fetch_result(out)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("offset", [0, 1])
def test_single_clip_pinned_buffers_equal_device_buffers(offset):
    for i, c in enumerate(_clips()):
        want = _device_run(c, 40 + i)
        rgb, mask = _pinned(c.rgb, offset), _pinned(c.mask, offset)
        out = _pinned(np.zeros_like(c.rgb), offset)
        with vi.Context(levels=c.levels, seed=40 + i) as ctx:
            ctx.upload(rgb, mask)
            ctx.run()
            ctx.fetch_result(out)
        assert (out.view(np.uint32) == want.view(np.uint32)).all(), (i, offset)
        # pageable numpy buffers (the copy engine)
        with vi.Context(levels=c.levels, seed=40 + i) as ctx:
            ctx.upload(c.rgb.copy(), c.mask.copy())
            ctx.run()
            got = ctx.fetch_result()
        assert (got.view(np.uint32) == want.view(np.uint32)).all(), i


@pytest.mark.parametrize("offset", [0, 1])
def test_batch_pinned_buffers_equal_device_buffers(offset):
    clips = _clips()
    want = [_device_run(c, 60 + i) for i, c in enumerate(clips)]
    items = [(_pinned(c.rgb, offset), _pinned(c.mask, offset), dict(levels=c.levels, seed=60 + i))
             for i, c in enumerate(clips)]
    outs = [_pinned(np.zeros_like(c.rgb), offset) for c in clips]
    with vi.Batch() as b:
        ids = b.add_many(items)
        b.run()
        for cid, o in zip(ids, outs):
            b.fetch(cid, o)
    for i, (o, w) in enumerate(zip(outs, want)):
        assert (o.view(np.uint32) == w.view(np.uint32)).all(), (i, offset)
