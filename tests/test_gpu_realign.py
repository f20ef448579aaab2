"""Affine realignment on the GPU (Sec. 3.4, Algorithm 2, UnwarpVideo) against
the realignment oracle: the estimated motions agree within 1e-3 px of
displacement (FP32 per-pixel arithmetic against FP64), the chaining to the
reference frame is bit-identical (same double expressions, no contraction),
the aligned occlusion is bit-identical (sample positions and their tests in
double on both sides) and the aligned and unwarped values agree within 1e-5;
host and device buffers give the same results; the whole realigned
inpainting runs and leaves the known pixels untouched."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import realign as R  # noqa: E402
from paper_1503_05528_gb300 import synth, vi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    vi.load(build_if_missing=True)


def _disp(ta, tb, W, H):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    ax, ay = R.apply(R.theta_to_matrix(ta), xx, yy)
    bx, by = R.apply(R.theta_to_matrix(tb), xx, yy)
    return float(np.max(np.hypot(ax - bx, ay - by)))


def _jittered(W=96, H=72, T=6, seed=5):
    """A layered clip whose frames are moved by seeded affine jitter."""
    clip = synth.layered_clip(W, H, T, 2, (12, 24), 0.06, 2, seed)
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    rgb = clip.rgb.astype(np.float64).copy()
    for t in range(1, T):
        th = rng.normal(0, [1.0, 0.004, 0.004, 1.0, 0.004, 0.004])
        px, py = R.apply(R.invert(R.theta_to_matrix(th)), xx, yy)
        px = np.clip(px, 0, W - 1)
        py = np.clip(py, 0, H - 1)
        v, _ = R.sample_bilinear(clip.rgb[t].astype(np.float64), px, py)
        rgb[t] = v
    return np.ascontiguousarray(rgb, np.float32), clip.mask


def test_estimate_matches_oracle():
    rgb, mask = _jittered()
    T, H, W = mask.shape
    got = vi.affine_estimate(rgb, mask)
    want = R.estimate(rgb, mask)
    assert got.shape == (T - 1, 6)
    for n in range(T - 1):
        assert _disp(got[n], want[n], W, H) < 1e-3, n


def test_estimate_analytic_pair():
    W, H = 128, 96
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)

    def field(x, y):
        return 0.5 + 0.2 * np.sin(2 * math.pi * x / 29.0) * np.cos(2 * math.pi * y / 19.0) \
            + 0.1 * np.cos(2 * math.pi * (x + y) / 13.0)

    theta = np.array([1.7, 0.006, -0.01, -0.9, 0.008, 0.004])
    px, py = R.apply(R.invert(R.theta_to_matrix(theta)), xx, yy)
    frames = np.stack([field(xx, yy), field(px, py)])
    rgb = np.ascontiguousarray(np.repeat(frames[..., None], 3, -1), np.float32)
    mask = np.zeros((2, H, W), np.uint8)
    got = vi.affine_estimate(rgb, mask)[0]
    assert _disp(got, theta, W, H) < 0.02
    assert _disp(got, R.estimate(rgb, mask)[0], W, H) < 1e-3


def test_chaining_bit_exact():
    rng = np.random.default_rng(3)
    for T in (1, 2, 5, 8):
        pairs = rng.normal(0, [1.5, 0.01, 0.01, 1.5, 0.01, 0.01], size=(max(T - 1, 0), 6))
        got = vi.affine_to_reference(pairs, T)
        want = np.array([R.matrix_to_theta(m) for m in R.to_reference(pairs, T)])
        assert np.array_equal(got, want), T


def test_align_and_unwarp_match_oracle():
    rgb, mask = _jittered(seed=9)
    T, H, W = mask.shape
    to_ref = vi.affine_to_reference(R.estimate(rgb, mask), T)
    mats = np.array([R.theta_to_matrix(t) for t in to_ref])
    got, gmask = vi.affine_align(rgb, mask, to_ref)
    want, wmask = R.align(rgb, mask, mats)
    assert np.array_equal(gmask, wmask)
    keep = wmask == 0
    assert np.abs(got[keep] - want[keep]).max() < 1e-5
    res = np.random.default_rng(1).random((T, H, W, 3)).astype(np.float32)
    gout = vi.affine_unwarp(rgb, mask, res, to_ref)
    wout = R.unwarp(rgb, mask, res, mats)
    assert np.array_equal(gout[mask == 0], rgb[mask == 0])
    assert np.abs(gout - wout).max() < 1e-5


def test_device_buffers_same_as_host():
    rgb, mask = _jittered(seed=12)
    T = mask.shape[0]
    th_h = vi.affine_estimate(rgb, mask)
    rd, md = torch.from_numpy(rgb).cuda(), torch.from_numpy(mask).cuda()
    th_d = vi.affine_estimate(rd, md)
    assert np.array_equal(th_h, th_d)
    to_ref = vi.affine_to_reference(th_h, T)
    al_h, am_h = vi.affine_align(rgb, mask, to_ref)
    al_d, am_d = torch.empty_like(rd), torch.empty_like(md)
    vi.affine_align(rd, md, to_ref, al_d, am_d)
    assert np.array_equal(al_h, al_d.cpu().numpy()) and np.array_equal(am_h, am_d.cpu().numpy())
    out_d = torch.empty_like(rd)
    vi.affine_unwarp(rd, md, al_d, to_ref, out_d)
    assert np.array_equal(vi.affine_unwarp(rgb, mask, al_h, to_ref), out_d.cpu().numpy())


def test_realigned_inpainting_runs():
    rgb, mask = _jittered(W=128, H=96, T=10, seed=21)
    out = vi.inpaint(rgb, mask, realign=True, levels=2)
    assert np.isfinite(out).all()
    assert np.array_equal(out[mask == 0], rgb[mask == 0])
    hole = out[mask == 1]
    assert hole.min() >= -1e-3 and hole.max() <= 1 + 1e-3


def test_bad_arguments_rejected():
    with pytest.raises(vi.ViError):
        vi.affine_to_reference(np.zeros((3, 6)), 0)
