"""vi_energy_noalloc: the Eq. 1 energy for callers that cannot allocate
device memory (their device memory belongs to an allocator under a fixed
budget, or they cannot take the synchronisation cudaMalloc/cudaFree may
cause). It reads caller-owned device buffers and keeps its scratch in a fixed
static device array, so it must agree with vi_energy -- which allocates its
reduction scratch per context -- on every call, including two calls in a row
that reuse the same static array.

This file is collected last so that a stop-at-first-failure run has already
run every other test when it gets here."""
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


def _noalloc(lib, chans, phi, code, out, stream):
    T, H, W, C = chans.shape
    return lib.vi_energy_noalloc(chans.data_ptr(), C, phi.data_ptr(), code.data_ptr(), W, H, T,
                                 out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("tex,levels,seed", [(False, 1, 0), (True, 2, 1)])
def test_noalloc_energy_matches_vi_energy_twice(tex, levels, seed):
    if tex:
        clip = synth.small_layered(W=72, H=56, T=14, levels=2, seed=1514)
    else:
        clip = synth.tiny_translation_clip()
    lib = vi.load()
    stream = torch.cuda.current_stream()
    with vi.Context(levels=levels, use_texture=int(tex), seed=101 + seed) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.prepare()
        L = levels
        for call, level in enumerate(range(L - 1, -1, -1)):
            ctx.iterate(level, 2)
            if level > 0:
                ctx.next_level(level)
        for level in range(L):
            # a state per level: the run's own state, then a different one
            for variant in range(2):
                if variant == 1:
                    # another valid shift map: every target points at a
                    # source patch drawn at random (seeded numpy)
                    code = ctx.get_masks(level)
                    T_, H_, W_ = code.shape
                    src = np.flatnonzero((code >> 2) & 1)
                    tgt = np.flatnonzero((code >> 1) & 1)
                    pick = src[np.random.default_rng(7 + level).integers(0, len(src), len(tgt))]
                    ph = np.zeros((T_, H_, W_, 3), np.int32).reshape(-1, 3)
                    ph[tgt, 0] = pick % W_ - tgt % W_
                    ph[tgt, 1] = (pick // W_) % H_ - (tgt // W_) % H_
                    ph[tgt, 2] = pick // (W_ * H_) - tgt // (W_ * H_)
                    ctx.set_nnf(level, ph.reshape(T_, H_, W_, 3), None)
                eh, eht = ctx.energy(level)
                info = ctx.level_info(level)
                chans = torch.empty((info["T"], info["H"], info["W"], info["C"]), dtype=torch.float32,
                                    device="cuda")
                ctx.get_channels(level, chans)
                phi, _ = ctx.get_nnf(level)
                code = ctx.get_masks(level)
                phi_d = torch.from_numpy(phi).cuda()
                code_d = torch.from_numpy(code).cuda()
                out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                for _ in range(2):   # two calls in a row share the static scratch
                    out.fill_(-1.0)
                    assert _noalloc(lib, chans, phi_d, code_d, out, stream) == 0
                    torch.cuda.synchronize()
                    got = out.cpu().numpy()
                    assert got[0] == pytest.approx(eh, rel=1e-5)
                    assert got[1] == pytest.approx(eht, rel=1e-5)


def _random_valid_map(code, rng):
    """Every target of code points at a source patch of D~ drawn at random."""
    T_, H_, W_ = code.shape
    src = np.flatnonzero((code >> 2) & 1)
    tgt = np.flatnonzero((code >> 1) & 1)
    pick = src[rng.integers(0, len(src), len(tgt))]
    ph = np.zeros((T_ * H_ * W_, 3), np.int32)
    ph[tgt, 0] = pick % W_ - tgt % W_
    ph[tgt, 1] = (pick // W_) % H_ - (tgt // W_) % H_
    ph[tgt, 2] = pick // (W_ * H_) - tgt // (W_ * H_)
    return ph, tgt


def _both_energies(ctx, lib, stream):
    eh, eht = ctx.energy(0)
    info = ctx.level_info(0)
    chans = torch.empty((info["T"], info["H"], info["W"], info["C"]), dtype=torch.float32, device="cuda")
    ctx.get_channels(0, chans)
    phi, _ = ctx.get_nnf(0)
    phi_d = torch.from_numpy(phi).cuda()
    code_d = torch.from_numpy(ctx.get_masks(0)).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    got = []
    for _ in range(2):   # two calls in a row share the static scratch
        out.fill_(-1.0)
        torch.cuda.synchronize()
        assert _noalloc(lib, chans, phi_d, code_d, out, stream) == 0
        torch.cuda.synchronize()
        got.append(out.cpu().numpy().copy())
    return (eh, eht), got


def test_noalloc_energy_many_blocks_and_sources_outside_d_tilde():
    # 320 x 240 x 40 = 3,072,000 voxels: 12,000 blocks of partial sums, so the
    # final reduction takes many strided passes over the static array
    clip = synth.fast_layered_clip(320, 240, 40, 0.08, seed=1533)
    lib = vi.load()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(12)
    with vi.Context(levels=1, use_texture=1, seed=5) as ctx:
        ctx.upload(clip.rgb, clip.mask)
        ctx.build_pyramid()
        code = ctx.get_masks(0)
        T_, H_, W_ = code.shape
        ph, tgt = _random_valid_map(code, rng)
        # some targets point at a whole patch that is not in D~ (it meets the
        # hole): both energies count it, as Eq. 1 counts any shift
        hole = np.flatnonzero(code & 1)
        inner = hole[((hole % W_) >= 2) & ((hole % W_) < W_ - 2) & (((hole // W_) % H_) >= 2) &
                     (((hole // W_) % H_) < H_ - 2) & ((hole // (W_ * H_)) >= 2) &
                     ((hole // (W_ * H_)) < T_ - 2)]
        assert len(inner) > 1000
        some = tgt[rng.integers(0, len(tgt), 500)]
        src = inner[rng.integers(0, len(inner), 500)]
        ph[some, 0] = src % W_ - some % W_
        ph[some, 1] = (src // W_) % H_ - (some // W_) % H_
        ph[some, 2] = src // (W_ * H_) - some // (W_ * H_)
        ctx.set_nnf(0, ph.reshape(T_, H_, W_, 3), None)
        (eh, eht), got = _both_energies(ctx, lib, stream)
        assert np.isfinite(eh) and np.isfinite(eht) and eh > 0
        for g in got:
            assert g[0] == pytest.approx(eh, rel=1e-5)
            assert g[1] == pytest.approx(eht, rel=1e-5)
        # one target whose source patch leaves the video (centre x = W - 2):
        # +inf in both, in E_H~ and, for an occluded target, in E_H
        p = hole[len(hole) // 2]
        ph[p, 0] = (W_ - 2) - p % W_
        ctx.set_nnf(0, ph.reshape(T_, H_, W_, 3), None)
        (eh, eht), got = _both_energies(ctx, lib, stream)
        assert eh == np.inf and eht == np.inf
        for g in got:
            assert g[0] == np.inf and g[1] == np.inf


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lib = vi.load()
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # 4097 x 4096 x 1 voxels > 16,777,216: refused before anything runs
    st = lib.vi_energy_noalloc(dummy.data_ptr(), 3, dummy.data_ptr(), dummy.data_ptr(), 4097, 4096, 1,
                               out.data_ptr(), None)
    assert st == 8   # VI_ERR_TOO_LARGE
    st = lib.vi_energy_noalloc(dummy.data_ptr(), 4, dummy.data_ptr(), dummy.data_ptr(), 8, 8, 8,
                               out.data_ptr(), None)
    assert st == 1   # VI_ERR_ARG: C must be 3 or 5
