"""Time slabs (vi_run_slabs): the inpainting with every level but the
coarsest split by frames over several contexts, with the boundary frames
copied between them, is identical to vi_run: the output bit for bit, the
iteration counts per level and the evaluation count. Covers one slab, even
and uneven splits, slabs of a single frame (a two-frame halo then spans
several slabs), the multi-radius search with propagation sub-sweeps, a
stream per slab ordered by events (the multi-device form, here with every
slab on this GPU), device buffers, and the argument checks."""
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


def _alone(c, **cfg):
    with vi.Context(**cfg) as ctx:
        ctx.upload(c.rgb, c.mask)
        ctx.run()
        return ctx.fetch_result(), ctx.stats()


def _check(c, n, devices=None, **cfg):
    want, ws = _alone(c, **cfg)
    got, gs, nbytes = vi.run_slabs(c.rgb, c.mask, n, devices=devices, **cfg)
    assert (got.view(np.uint32) == want.view(np.uint32)).all()
    assert gs["outer"] == ws["outer"]
    assert gs["evals"] == ws["evals"]
    assert (nbytes > 0) == (n > 1 and cfg["levels"] > 1)
    return nbytes


@pytest.mark.parametrize("n", [1, 2, 3, 7, 14])
def test_two_levels_every_split(n):
    c = synth.small_layered(W=72, H=56, T=14, levels=2, seed=1701)
    _check(c, n, levels=2, seed=91, clip=3)


@pytest.mark.parametrize("n", [2, 4])
def test_three_levels(n):
    c = synth.layered_clip(96, 64, 20, 2, (10, 20), 0.08, 3, 1702)
    _check(c, n, levels=3, seed=92)


def test_uneven_split_and_search_options():
    c = synth.small_layered(W=64, H=48, T=13, levels=2, seed=1703)
    _check(c, 3, levels=2, seed=93, rs_mode=1, sub_sweeps=2)
    _check(c, 5, levels=2, seed=94, lanes_per_target=32)


@pytest.mark.parametrize("n", [2, 3, 14])
def test_a_stream_per_slab(n):
    # the multi-device form (a context, stream and event per slab, peer
    # copies ordered by events) with every slab on this GPU: the same result,
    # and the same bytes exchanged as on one shared stream
    c = synth.small_layered(W=72, H=56, T=14, levels=2, seed=1706)
    nb = _check(c, n, devices=[0] * n, levels=2, seed=96, clip=1)
    _, _, nb1 = vi.run_slabs(c.rgb, c.mask, n, levels=2, seed=96, clip=1)
    assert nb == nb1


def test_device_buffers():
    c = synth.small_layered(W=72, H=56, T=14, levels=2, seed=1704)
    want, _ = _alone(c, levels=2, seed=95)
    rgb, mask = torch.from_numpy(c.rgb).cuda(), torch.from_numpy(c.mask).cuda()
    out = torch.empty_like(rgb)
    stream = torch.cuda.current_stream()
    vi.run_slabs(rgb, mask, 3, out=out, stream=stream.cuda_stream, levels=2, seed=95)
    stream.synchronize()
    assert (out.cpu().numpy().view(np.uint32) == want.view(np.uint32)).all()


def test_bad_arguments():
    c = synth.small_layered(W=48, H=40, T=6, levels=1, seed=1705)
    for n, cfg in [(0, {}), (7, {}), (17, {}), (2, {"storage": 1}), (2, {"time_subsample": 1}),
                   (2, {"devices": [0, 999]})]:
        with pytest.raises(vi.ViError):
            vi.run_slabs(c.rgb, c.mask, n, levels=1, **cfg)
