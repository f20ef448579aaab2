"""Pins for the realignment oracle (Sec. 3.4, Algorithm 2, UnwarpVideo of
Algorithm 4): the dominant affine motion of frames generated from an
analytic image moved by a known affine map is recovered, also with an
outlier region moving otherwise and with a garbage-filled occluded region;
the map algebra (inverse, composition, chaining to the reference frame);
identity and integer-translation warps are exact; warping and unwarping are
mutual inverses; and the layered generator's own camera drift is recovered
between real frames."""
import math

import numpy as np
import pytest

from oracle import realign as R
from paper_1503_05528_gb300 import synth


def _field(x, y):
    """A smooth analytic image (periods 11 to 37 px)."""
    return (0.5 + 0.15 * np.sin(2 * math.pi * x / 23.0 + 0.3) * np.cos(2 * math.pi * y / 17.0)
            + 0.1 * np.sin(2 * math.pi * (x + 2 * y) / 37.0) + 0.07 * np.cos(2 * math.pi * (x - y) / 11.0))


def _pair(theta, W=96, H=72):
    """Frame 1 = field; frame 2 shows each point p of frame 1 at A(p), i.e.
    frame2(q) = field(A^-1(q)) exactly."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    I1 = _field(xx, yy)
    px, py = R.apply(R.invert(R.theta_to_matrix(theta)), xx, yy)
    I2 = _field(px, py)
    return I1, I2


def _disp_err(ta, tb, W=96, H=72):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    ax, ay = R.apply(R.theta_to_matrix(ta), xx, yy)
    bx, by = R.apply(R.theta_to_matrix(tb), xx, yy)
    return float(np.max(np.hypot(ax - bx, ay - by)))


THETAS = [np.array([1.3, 0.0, 0.0, -0.7, 0.0, 0.0]),                   # translation
          np.array([0.8, 0.01, -0.008, 0.4, 0.006, 0.012]),            # general affine
          np.array([-2.1, -0.004, 0.02, 1.6, -0.02, -0.004])]          # rotation-like


@pytest.mark.parametrize("k", range(len(THETAS)))
def test_recovers_known_affine_motion(k):
    I1, I2 = _pair(THETAS[k])
    z = np.zeros_like(I1, np.uint8)
    est = R.estimate_pair(I1, z, I2, z)
    assert _disp_err(est, THETAS[k]) < 0.02


def test_identity_motion():
    I1, _ = _pair(np.zeros(6))
    z = np.zeros_like(I1, np.uint8)
    est = R.estimate_pair(I1, z, I1.copy(), z)
    assert np.abs(est).max() < 1e-9


def test_robust_to_an_outlier_region():
    theta = THETAS[1]
    I1, I2 = _pair(theta)
    # a square of frame 2 replaced by content moving otherwise (about 9% of it)
    I2[20:42, 30:58] = _field(np.arange(30, 58)[None, :] * 1.7, np.arange(20, 42)[:, None] * 0.6 + 5.0)
    z = np.zeros_like(I1, np.uint8)
    est = R.estimate_pair(I1, z, I2, z)
    assert _disp_err(est, theta) < 0.05
    ls = R.estimate_pair(I1, z, I2, z, iters=1, levels=1)      # one least-squares step is pulled off
    assert _disp_err(ls, theta) > _disp_err(est, theta)


def test_occluded_pixels_take_no_part():
    theta = THETAS[0]
    I1, I2 = _pair(theta)
    o1 = np.zeros_like(I1, np.uint8)
    o2 = np.zeros_like(I1, np.uint8)
    o1[30:50, 10:40] = 1
    I1[o1 == 1] = 7.0                  # garbage under the occlusion
    o2[10:20, 60:80] = 1
    I2[o2 == 1] = -3.0
    est = R.estimate_pair(I1, o1, I2, o2)
    assert _disp_err(est, theta) < 0.02


def test_map_algebra():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = rng.normal(0, [2, 0.02, 0.02, 2, 0.02, 0.02])
        b = rng.normal(0, [2, 0.02, 0.02, 2, 0.02, 0.02])
        ma, mb = R.theta_to_matrix(a), R.theta_to_matrix(b)
        np.testing.assert_allclose(R.compose(ma, R.invert(ma)), R.theta_to_matrix(np.zeros(6)), atol=1e-12)
        x, y = rng.uniform(0, 100, 2)
        np.testing.assert_allclose(R.apply(R.compose(mb, ma), x, y), R.apply(mb, *R.apply(ma, x, y)), atol=1e-9)
        np.testing.assert_allclose(R.matrix_to_theta(ma), a, atol=1e-15)


def test_chaining_to_the_reference_frame():
    # translations chain by adding; N_m = floor(N_f / 2) counted from 1
    T = 7
    steps = np.zeros((T - 1, 6))
    steps[:, 0] = np.arange(1, T)           # frame n moves by n + 1 px in x to frame n + 1
    steps[:, 3] = -0.5
    to_ref = R.to_reference(steps, T)
    r = R.reference_frame(T)
    assert r == 2
    for n in range(T):
        want_x = sum(steps[m, 0] for m in range(n, r)) - sum(steps[m, 0] for m in range(r, n))
        want_y = -0.5 * (r - n)
        np.testing.assert_allclose(R.matrix_to_theta(to_ref[n]), [want_x, 0, 0, want_y, 0, 0], atol=1e-12)
    assert R.reference_frame(1) == 0 and R.reference_frame(2) == 0 and R.reference_frame(60) == 29


def test_identity_and_integer_warps():
    rng = np.random.default_rng(2)
    T, H, W = 3, 20, 24
    rgb = rng.random((T, H, W, 3))
    mask = (rng.random((T, H, W)) < 0.1).astype(np.uint8)
    ident = R.to_reference(np.zeros((T - 1, 6)), T)
    out, occ = R.align(rgb, mask, ident)
    assert np.array_equal(out, rgb) and np.array_equal(occ, mask)
    # the reference is frame 0, and frame 0 moves by (+2, -1) into frame 1
    steps = np.zeros((T - 1, 6))
    steps[0] = [2, 0, 0, -1, 0, 0]
    assert R.reference_frame(T) == 0
    out, occ = R.align(rgb, mask, R.to_reference(steps, T))
    # frame 1 maps to the reference by the inverse step: it reads frame 1 at q + (2, -1)
    assert np.array_equal(out[1][1:, :W - 2], rgb[1][:H - 1, 2:])
    assert occ[1][:, W - 2:].all() and occ[1][0].all()
    assert np.array_equal(occ[1][1:, :W - 2], mask[1][:H - 1, 2:])


def test_align_then_unwarp_restores_smooth_content():
    T, H, W = 5, 48, 64
    theta = np.array([0.6, 0.004, -0.003, -0.4, 0.002, 0.005])
    steps = np.tile(theta, (T - 1, 1))
    to_ref = R.to_reference(steps, T)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    rgb = np.stack([np.stack([_field(xx + 3 * t, yy - t) * s for s in (1.0, 0.9, 0.8)], -1)
                    for t in range(T)])
    mask = np.zeros((T, H, W), np.uint8)
    mask[:, 18:30, 24:40] = 1
    al, occ = R.align(rgb, mask, to_ref)
    # the "inpainting" knows the truth: it fills the aligned hole with the
    # aligned ground truth; unwarping must give the ground truth back
    truth_al, _ = R.align(rgb, np.zeros_like(mask), to_ref)
    filled = np.where(occ[..., None] == 1, truth_al, al)
    out = R.unwarp(np.where(mask[..., None] == 1, 0.0, rgb), mask, filled, to_ref)
    err = np.abs(out - rgb)[mask == 1]
    # two bilinear resamplings of content with 11 px periods: a few percent at most
    assert err.max() < 0.05 and err.mean() < 0.01
    assert np.array_equal(out[mask == 0], rgb[mask == 0])
    # a planted mistake (unwarping with the inverse maps) is far off
    bad = R.unwarp(np.where(mask[..., None] == 1, 0.0, rgb), mask, filled,
                   np.array([R.invert(m) for m in to_ref]))
    assert np.abs(bad - rgb)[mask == 1].mean() > 5 * err.mean()


def test_recovers_the_generator_camera_drift():
    # frames of the layered generator without sprites: the background is
    # sampled at R(t)(p - c) + c + d t + margin, so frame t+1 shows the point
    # p of frame t at R(t+1)^-1 (R(t)(p - c) - d) + c: an exact affine motion
    # (up to the generator's own bilinear resampling)
    W, H, T = 96, 72, 3
    clip = synth.layered_clip(W, H, T, 0, (10, 20), 0.05, 1, 4242)
    I = R.grey(clip.rgb)
    z = np.zeros((H, W), np.uint8)
    est = R.estimate_pair(I[0], z, I[1], z)
    # the true motion, from the generator's parameters
    g = np.random.default_rng(4242)
    margin = 48
    bh, bw = H + 2 * margin, W + 2 * margin
    for sig in (1.0, 4.0, 16.0):
        synth.smooth_noise(g, bh, bw, sig)
    dtx, dty = g.uniform(-0.5, 0.5), g.uniform(-0.5, 0.5)
    drot, dscale = g.uniform(-0.002, 0.002), g.uniform(-0.001, 0.001)

    def rmat(t):
        s = 1.0 + dscale * t
        return np.array([[math.cos(drot * t) * s, -math.sin(drot * t) * s],
                         [math.sin(drot * t) * s, math.cos(drot * t) * s]])

    c = np.array([W / 2.0, H / 2.0])
    A = np.linalg.inv(rmat(1)) @ rmat(0)
    b = c - A @ c - np.linalg.inv(rmat(1)) @ np.array([dtx, dty])
    true = np.array([b[0], A[0, 0] - 1, A[0, 1], b[1], A[1, 0], A[1, 1] - 1])
    assert _disp_err(est, true, W, H) < 0.05
