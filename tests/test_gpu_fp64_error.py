"""The error of each output of the GPU path against the oracle run in FP64
(distances, stored distances, decisions, weights and sums in double; the
video between steps in FP32, as the input is): shift maps, distances, the
vote and the final step of Eq. 6, and a whole inpainting. FP16 storage
takes the FP32 path's decisions and votes from the FP32 channels, so its
outputs are the FP32 path's bit for bit (tests/test_gpu_fp16.py checks
that) and so are its errors; both storages run here. The figures are printed
(pytest -s) and bounded:

  - the shift map after one search agrees with the FP64 search on at least
    99% of the targets (FP32 rounding decides only near-ties);
  - where the shifts agree, the FP32 distance is within 2e-5 relative of the
    FP64 one (at most 625 rounded terms);
  - the FP32 vote of a given shift map is within 1e-4 of the FP64 vote of the
    same shift map (the parity bar for voxels);
  - a whole inpainting's energy of Eq. 1 is within 2% of the FP64 run's."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1503_05528_gb300 import synth, vi  # noqa: E402

pytestmark = pytest.mark.gpu

SUB = 2

CASES = {
    "layered_72x56x14": lambda: synth.small_layered(W=72, H=56, T=14, levels=2, seed=1514),
    "fast_160x120x20": lambda: synth.fast_layered_clip(160, 120, 20, 0.08, seed=1535),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


def _d2_f64(x, phi, mask):
    out = np.full(mask.shape, np.inf, np.float64)
    for (t, y, xx) in zip(*np.nonzero(mask)):
        dx, dy, dt = phi[t, y, xx]
        out[t, y, xx] = O.dist(x, (xx, y, t), (xx + dx, y + dy, t + dt), fp64=True)
    return out


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("storage", [0, 2])
def test_step_outputs_against_fp64(case, storage):
    clip = CASES[case]()
    lv = O.build_pyramid(clip.rgb, clip.mask, 1, True)[0]
    rng = np.random.default_rng(9)
    x = lv.x.copy()
    h = lv.hole.astype(bool)
    x[h] = rng.random((int(h.sum()), 5), dtype=np.float32) * np.float32(0.8) + np.float32(0.1)
    phi0 = O.init_nnf(lv.htilde, lv.dtilde, (71, 0), O.tag(O.PURPOSE_INIT, 0))
    t = lv.htilde == 1
    with vi.Context(levels=1, use_texture=1, seed=71, sub_sweeps=SUB, storage=storage) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.build_pyramid()
        ctx.set_channels(0, x)
        ctx.set_nnf(0, phi0, np.full(lv.hole.shape, np.inf, np.float32))
        ctx.ann(0, 0)
        gphi, gd2 = ctx.get_nnf(0)
        ctx.reconstruct(0)
        gx = ctx.get_channels(0)
        ctx.final()
        gf = ctx.get_channels(0)
    # the FP64 search from the same state
    p64 = phi0.copy()
    d64 = np.full(lv.hole.shape, np.inf, np.float64)
    O.ann(x, lv.htilde, lv.dtilde, p64, d64, n_pm=10, key=(71, 0), tag_base=O.tag(O.PURPOSE_SEARCH, 0, 0),
          sub_sweeps=SUB)
    agree = (gphi == p64).all(axis=-1) & t
    nnf_disagree = 1.0 - agree.sum() / t.sum()
    rel = np.abs(gd2[agree].astype(np.float64) - d64[agree]) / np.maximum(d64[agree], 1e-30)
    # the FP64 vote and final step of the GPU's own shift map (their
    # arithmetic alone), and of the FP64 search's shift map (end of the step)
    gd64 = _d2_f64(x, gphi, t)
    v64, _ = O.vote(x, lv.hole, lv.htilde, gphi, gd64, weighted=True, n_diff=3)
    dv = np.abs(gx[h] - v64[h])
    o64, _ = O.vote(x, lv.hole, lv.htilde, p64, d64, weighted=True, n_diff=3)
    dstep = np.abs(gx[h][:, :3] - o64[h][:, :3])
    f64 = O.final(v64, lv.hole, gphi, gd64)
    # Eq. 6 copies one voxel: the fraction of occluded voxels whose copy
    # source differs from the FP64 argmin of the same distances
    final_diff = float(np.mean((gf[h][:, :3] != f64[h][:, :3]).any(axis=-1)))
    print(f"\n{case} storage {storage}: targets {int(t.sum())}; shift-map disagreement {nnf_disagree:.2e}; "
          f"d2 rel. error max {rel.max():.2e} mean {rel.mean():.2e}; "
          f"vote (same shifts) max {dv.max():.2e} mean {dv.mean():.2e}; "
          f"vote (each side's search) RGB max {dstep.max():.2e} mean {dstep.mean():.2e}; "
          f"final step copies differing {final_diff:.2e}")
    assert nnf_disagree <= 0.01
    assert rel.max() <= 2e-5
    assert dv.max() <= 1e-4 * math.sqrt(50.0) and dv[:, :3].max() <= 1e-4


@pytest.mark.parametrize("storage", [0, 2])
def test_whole_inpainting_against_fp64(storage):
    clip = CASES["layered_72x56x14"]()
    L = 2
    with vi.Context(levels=L, use_texture=1, seed=73, storage=storage) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.prepare()
        for level in range(L - 1, -1, -1):
            ctx.iterate(level)
            if level > 0:
                ctx.next_level(level)
        gx = ctx.get_channels(0)
        gphi, _ = ctx.get_nnf(0)
        outer = ctx.stats()["outer"][:L]
        ctx.final()
        gout = ctx.fetch_result()
    prm = O.Params(seed=73, sub_sweeps=SUB, fp64=True, fixed_outer=[outer[1], outer[0]])
    out64, pyr, before = O.inpaint(clip.rgb, clip.mask, L, True, prm, return_levels=True)
    lv = pyr[0]
    e_gpu = O.energy(gx, lv.hole, lv.htilde, gphi)
    e_64 = O.energy(before, lv.hole, lv.htilde, lv.phi)
    h = clip.mask == 1
    d = np.abs(gout[h] - out64[h])
    mse = float(np.mean((gout[h] - out64[h]) ** 2))
    psnr = 10 * math.log10(1.0 / mse) if mse > 0 else float("inf")
    agree = float(np.mean((gphi == lv.phi).all(axis=-1)[lv.htilde == 1]))
    print(f"\nwhole inpainting, storage {storage}: E_H {e_gpu[0]:.6g} vs FP64 {e_64[0]:.6g} "
          f"(rel {e_gpu[0] / e_64[0] - 1:+.2e}); E_H~ rel {e_gpu[1] / e_64[1] - 1:+.2e}; "
          f"final shift maps agree on {agree:.4f} of targets; output vs FP64 output: max {d.max():.3g}, "
          f"mean {d.mean():.3g}, PSNR {psnr:.1f} dB")
    assert e_gpu[0] <= 1.02 * e_64[0] and e_gpu[1] <= 1.02 * e_64[1]
