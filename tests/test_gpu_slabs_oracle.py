"""Time slabs (vi_run_slabs) against the oracle rather than against vi_run:
a whole inpainting split by frames over 2 and 3 contexts, on two- and
three-level clips, is compared voxel by voxel with the oracle's inpainting
(Algorithm 4 with the Jacobi schedule, the same propagation sweeps, Philox
key and counter word), its per-level iteration counts fixed to the ones the
slabbed run's stopping rule chose. Every search decision of the GPU path is
the oracle's (bit-exact shift maps step by step); the votes differ by FP32
against FP64 rounding, which could turn a later near-tie, so the bar is: at
least 99.9% of the occluded voxels within 1e-4 and the mean difference below
1e-5. The slabs' boundary exchange is also checked on CPU ranks against the
oracle (tests/test_slabs_cpu_ranks.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1503_05528_gb300 import synth, vi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


CASES = [
    ("72x56x14_L2", lambda: synth.small_layered(W=72, H=56, T=14, levels=2, seed=1701), 2, 3, 91),
    ("72x56x14_L2", lambda: synth.small_layered(W=72, H=56, T=14, levels=2, seed=1701), 2, 2, 95),
    ("96x64x20_L3", lambda: synth.layered_clip(96, 64, 20, 2, (10, 20), 0.08, 3, 1702), 3, 3, 92),
]


@pytest.mark.parametrize("name,make,levels,n,seed", CASES)
def test_slabbed_inpainting_matches_the_oracle(name, make, levels, n, seed):
    c = make()
    cfg = vi.default_config()
    got, st, nbytes = vi.run_slabs(c.rgb, c.mask, n, levels=levels, seed=seed, clip=2)
    assert nbytes > 0
    outer = st["outer"][:levels]
    prm = O.Params(seed=seed, clip=2, sub_sweeps=cfg.sub_sweeps,
                   fixed_outer=[outer[lv] for lv in range(levels - 1, -1, -1)])
    want = O.inpaint(c.rgb, c.mask, levels, True, prm)
    h = c.mask == 1
    d = np.abs(got[h] - want[h]).max(axis=-1)
    frac = float(np.mean(d <= 1e-4))
    print(f"\n{name}, {n} slabs: outer {outer}; voxels within 1e-4: {frac:.5f}; "
          f"mean |diff| {float(d.mean()):.2e}; max {float(d.max()):.2e}")
    assert frac >= 0.999
    assert float(d.mean()) <= 1e-5
    known = ~h
    assert (got[known] == c.rgb[known]).all()
