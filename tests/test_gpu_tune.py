"""Lanes-per-target autotuning: the table fills on first use, exports and
imports as text, rejects malformed lines, and whatever lane counts it holds
the results stay bit-identical (the lane count is a speed choice only)."""
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


def _run(clip):
    with vi.Context(levels=clip.levels, seed=5, clip=1) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.run()
        return ctx.fetch_result(), ctx.get_nnf(0)[0]


def _parse(text):
    return [tuple(int(v) for v in line.split()) for line in text.splitlines() if line.strip()]


def test_table_roundtrip_and_results_independent_of_choices():
    clip = synth.small_layered(W=96, H=72, T=16, levels=2, seed=1901)
    out0, phi0 = _run(clip)
    table = vi.tune_export()
    rows = _parse(table)
    assert rows and all(len(r) == 6 and r[5] in (1, 2, 4, 8, 32) for r in rows)
    assert all(r[5] != 32 or r[1] in (0, 1) for r in rows)   # warp-shared: the step kernels only
    try:
        for G in (8, 1, 2, 32):
            # force every known bucket to G (the warp-shared form where it
            # exists): the next run must not change
            vi.tune_import("".join(f"{d} {f} {c} {h} {b} {G if G != 32 or f in (0, 1) else 1}\n"
                                   for d, f, c, h, b, _ in rows))
            assert all(r[5] == (G if G != 32 or r[1] in (0, 1) else 1)
                       for r in _parse(vi.tune_export()) if r[:5] in {x[:5] for x in rows})
            out, phi = _run(clip)
            assert (out.view(np.uint32) == out0.view(np.uint32)).all()
            assert (phi == phi0).all()
    finally:
        vi.tune_import(table)
    assert _parse(vi.tune_export()) == rows


@pytest.mark.parametrize("bad", ["0 0 1 0 77", "0 9 1 0 77 2", "0 0 1 0 77 3", "0 2 1 0 77 32", "x y z"])
def test_malformed_import_rejected(bad):
    before = vi.tune_export()
    with pytest.raises(vi.ViError):
        vi.tune_import(bad + "\n")
    assert vi.tune_export() == before
