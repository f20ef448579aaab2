"""Seeded synthetic inputs: layered-motion videos and occlusion tubes.

This module only *makes inputs*. It holds none of the inpainting method's
arithmetic (no patch distance, search, vote or pyramid step), so both the
CUDA path and the CPU oracle may consume what it produces.

Every generator is a pure function of its arguments and a seed
(``numpy.random.default_rng``). Videos are float32 ``[T][H][W][3]`` in [0, 1];
masks are uint8 ``[T][H][W]`` with 1 = occluded (the set H of Sec. 2).

The workloads stand in for the paper's real clips (Table 1), which are not
available: a textured background under a slow affine camera drift, textured
sprites on linear paths, an optional dynamic-texture region (AR(1) noise, the
"Waves"-like case of Fig. 7) and a moving elliptical occlusion tube.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1503


@dataclass
class Clip:
    """One synthetic inpainting job."""

    name: str
    rgb: np.ndarray            # float32 [T][H][W][3], values under the mask included
    mask: np.ndarray           # uint8 [T][H][W], 1 = occluded
    levels: int                # pyramid levels L
    use_texture: bool          # texture-feature channels on (C = 5) or off (C = 3)
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        T, H, W = self.mask.shape
        return W, H, T


def smooth_noise(rng, height, width, sigma, channels=3, lo=0.1, hi=0.9):
    """Gaussian white noise blurred with a periodic Gaussian of std ``sigma`` px,
    each channel affinely normalised to [lo, hi]. float64 [height][width][channels]."""
    n = rng.standard_normal((channels, height, width))
    fy = np.fft.fftfreq(height)[:, None]
    fx = np.fft.fftfreq(width)[None, :]
    transfer = np.exp(-2.0 * (math.pi ** 2) * (sigma ** 2) * (fx ** 2 + fy ** 2))
    out = np.real(np.fft.ifft2(np.fft.fft2(n) * transfer[None]))
    mn = out.min(axis=(1, 2), keepdims=True)
    mx = out.max(axis=(1, 2), keepdims=True)
    out = lo + (hi - lo) * (out - mn) / np.maximum(mx - mn, 1e-12)
    return np.ascontiguousarray(np.moveaxis(out, 0, -1))


def _bilinear(img, sx, sy):
    """Sample img [h][w][c] at float coords (clamped to the border)."""
    h, w = img.shape[:2]
    sx = np.clip(sx, 0.0, w - 1.000001)
    sy = np.clip(sy, 0.0, h - 1.000001)
    x0 = np.floor(sx).astype(np.int64)
    y0 = np.floor(sy).astype(np.int64)
    fx = (sx - x0)[..., None]
    fy = (sy - y0)[..., None]
    a = img[y0, x0]
    b = img[y0, x0 + 1]
    c = img[y0 + 1, x0]
    d = img[y0 + 1, x0 + 1]
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy


def translating_texture(W, H, T, sigma=2.0, seed=BASE_SEED + 1, speed=1):
    """u(x, y, t) = f((x - speed*t) mod W, y): a periodic smooth texture sliding
    ``speed`` px per frame. Returns float32 [T][H][W][3]."""
    rng = np.random.default_rng(seed)
    f = smooth_noise(rng, H, W, sigma)
    xs = np.arange(W)
    frames = [f[:, (xs - speed * t) % W, :] for t in range(T)]
    return np.ascontiguousarray(np.stack(frames), dtype=np.float32)


def box_mask(W, H, T, x0, x1, y0, y1, t0, t1):
    """uint8 mask with the inclusive box [x0,x1]x[y0,y1]x[t0,t1] occluded."""
    m = np.zeros((T, H, W), np.uint8)
    m[t0:t1 + 1, y0:y1 + 1, x0:x1 + 1] = 1
    return m


def tiny_translation_clip():
    """32x32 px x 8 frames, smooth-noise texture (sigma 2 px) translating
    1 px/frame, centred 8x8x4 box occlusion, 1 level, RGB only."""
    W, H, T = 32, 32, 8
    rgb = translating_texture(W, H, T, sigma=2.0, seed=BASE_SEED + 1)
    mask = box_mask(W, H, T, 12, 19, 12, 19, 2, 5)
    return Clip("tiny_32x32x8", rgb, mask, levels=1, use_texture=False,
                meta={"outer_iters": 10})


def _ellipse_tube(W, H, T, frac, rng, axis_ratio=1.5):
    """Moving elliptical occlusion tube: per-frame ellipse of area frac*W*H,
    axis ratio ``axis_ratio``, centre moving linearly across the middle third."""
    b = math.sqrt(frac * W * H / (axis_ratio * math.pi))
    a = axis_ratio * b
    cx0, cx1 = W / 3.0, 2.0 * W / 3.0
    if rng.random() < 0.5:
        cx0, cx1 = cx1, cx0
    cy0 = H / 2.0 + rng.uniform(-0.08, 0.08) * H
    cy1 = H / 2.0 + rng.uniform(-0.08, 0.08) * H
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    mask = np.zeros((T, H, W), np.uint8)
    for t in range(T):
        s = t / max(T - 1, 1)
        cx = cx0 + (cx1 - cx0) * s
        cy = cy0 + (cy1 - cy0) * s
        inside = ((xx + 0.5 - cx) / a) ** 2 + ((yy + 0.5 - cy) / b) ** 2 <= 1.0
        mask[t][inside] = 1
    return mask


def layered_clip(W, H, T, n_sprites, sprite_px, hole_frac, levels, seed,
                 dynamic_texture=False, name=None, use_texture=True):
    """Layered synthetic video: drifting textured background, ``n_sprites``
    textured ellipses (diameters in ``sprite_px``) on linear paths at 1-3 px per
    frame (z-ordered by index), an optional AR(1) dynamic-texture rectangle
    (about 15% of the frame) and a moving elliptical occlusion tube of
    ``hole_frac`` of the voxels."""
    rng = np.random.default_rng(seed)
    margin = 48
    bh, bw = H + 2 * margin, W + 2 * margin
    bg = (0.2 * smooth_noise(rng, bh, bw, 1.0) + 0.35 * smooth_noise(rng, bh, bw, 4.0)
          + 0.45 * smooth_noise(rng, bh, bw, 16.0))
    mn, mx = bg.min(), bg.max()
    bg = 0.1 + 0.8 * (bg - mn) / (mx - mn)

    # Camera drift: per-frame increments of translation / rotation / scale.
    dtx = rng.uniform(-0.5, 0.5)
    dty = rng.uniform(-0.5, 0.5)
    drot = rng.uniform(-0.002, 0.002)
    dscale = rng.uniform(-0.001, 0.001)

    sprites = []
    for _ in range(n_sprites):
        d = rng.uniform(sprite_px[0], sprite_px[1])
        ra = d / 2.0
        rb = ra * rng.uniform(0.6, 1.0)
        side = int(math.ceil(2 * ra)) + 4
        tex = smooth_noise(rng, side, side, rng.uniform(1.0, 3.0),
                           lo=rng.uniform(0.05, 0.4), hi=rng.uniform(0.6, 0.95))
        speed = rng.uniform(1.0, 3.0)
        ang = rng.uniform(0, 2 * math.pi)
        x0 = rng.uniform(0.1 * W, 0.9 * W)
        y0 = rng.uniform(0.1 * H, 0.9 * H)
        sprites.append((ra, rb, tex, x0, y0, speed * math.cos(ang), speed * math.sin(ang)))

    dyn = None
    if dynamic_texture:
        rw, rh = int(0.45 * W), int(0.33 * H)
        rx = int(rng.uniform(0.05, 0.5) * W)
        ry = int(rng.uniform(0.05, 0.6) * H)
        tint = rng.uniform(0.3, 0.7, size=3)
        fy = np.fft.fftfreq(rh)[:, None]
        fx = np.fft.fftfreq(rw)[None, :]
        transfer = np.exp(-2.0 * (math.pi ** 2) * (1.5 ** 2) * (fx ** 2 + fy ** 2))
        state = rng.standard_normal((rh, rw))
        dyn = (rx, ry, rw, rh, tint, transfer, state)

    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cx, cy = W / 2.0, H / 2.0
    out = np.empty((T, H, W, 3), np.float32)
    for t in range(T):
        ang = drot * t
        sc = 1.0 + dscale * t
        ca, sa = math.cos(ang) * sc, math.sin(ang) * sc
        px, py = xx - cx, yy - cy
        sx = ca * px - sa * py + cx + dtx * t + margin
        sy = sa * px + ca * py + cy + dty * t + margin
        frame = _bilinear(bg, sx, sy)
        if dyn is not None:
            rx, ry, rw, rh, tint, transfer, state = dyn
            if t > 0:
                state = 0.9 * state + math.sqrt(1.0 - 0.81) * rng.standard_normal(state.shape)
                dyn = (rx, ry, rw, rh, tint, transfer, state)
            field_ = np.real(np.fft.ifft2(np.fft.fft2(state) * transfer))
            field_ = field_ / (np.abs(field_).max() + 1e-12)
            frame[ry:ry + rh, rx:rx + rw, :] = np.clip(tint[None, None, :] + 0.25 * field_[..., None], 0, 1)
        for (ra, rb, tex, x0, y0, vx, vy) in sprites:
            scx = x0 + vx * t
            scy = y0 + vy * t
            ins = ((xx + 0.5 - scx) / ra) ** 2 + ((yy + 0.5 - scy) / rb) ** 2 <= 1.0
            if not ins.any():
                continue
            side = tex.shape[0]
            tx = np.clip((xx[ins] - scx + side / 2.0).astype(np.int64), 0, side - 1)
            ty = np.clip((yy[ins] - scy + side / 2.0).astype(np.int64), 0, side - 1)
            frame[ins] = tex[ty, tx]
        out[t] = frame.astype(np.float32)
    np.clip(out, 0.0, 1.0, out=out)
    mask = _ellipse_tube(W, H, T, hole_frac, rng)
    return Clip(name or f"layered_{W}x{H}x{T}", out, mask, levels=levels,
                use_texture=use_texture,
                meta={"seed": seed, "n_sprites": n_sprites, "hole_frac": hole_frac,
                      "dynamic_texture": dynamic_texture})


def layered_320x240x60():
    """320x240 px x 60 frames, 3 sprites of 20-50 px, 8% occlusion tube,
    4 pyramid levels, colour + 2 texture-feature channels."""
    return layered_clip(320, 240, 60, 3, (20, 50), 0.08, 4, BASE_SEED + 2,
                        name="layered_320x240x60")


def layered_1280x720x100():
    """1280x720 px x 100 frames, 6 sprites of 40-160 px, AR(1) dynamic-texture
    region, 5% occlusion tube, 5 pyramid levels."""
    return layered_clip(1280, 720, 100, 6, (40, 160), 0.05, 5, BASE_SEED + 3,
                        dynamic_texture=True, name="layered_1280x720x100")


def small_layered(W=72, H=56, T=14, levels=2, seed=BASE_SEED + 11, hole_frac=0.08,
                  n_sprites=2, dynamic_texture=False):
    """A small layered clip for parity cases that span several tiles."""
    return layered_clip(W, H, T, n_sprites, (10, 20), hole_frac, levels, seed,
                        dynamic_texture=dynamic_texture, name=f"layered_{W}x{H}x{T}")


def fast_layered_clip(W, H, T, hole_frac, seed, n_sprites=2, name=None):
    """A cheaper layered clip for load tests: a two-octave smooth-noise
    background under an integer camera drift (whole-pixel shifts, no
    resampling), textured rectangles on integer linear paths, and the moving
    elliptical occlusion tube of layered_clip. Pyramid levels by the rule of
    Sec. 3.6 (levels = 0)."""
    rng = np.random.default_rng(seed)
    bg = (0.4 * smooth_noise(rng, H, W, 2.0) + 0.6 * smooth_noise(rng, H, W, 8.0)).astype(np.float32)
    mn, mx = bg.min(), bg.max()
    bg = (0.1 + 0.8 * (bg - mn) / (mx - mn)).astype(np.float32)
    vx, vy = int(rng.integers(-1, 2)), int(rng.integers(-1, 2))
    sprites = []
    for _ in range(n_sprites):
        sw, sh = int(rng.integers(W // 12 + 4, W // 5 + 5)), int(rng.integers(H // 12 + 4, H // 5 + 5))
        tex = smooth_noise(rng, sh, sw, 1.5, lo=0.05, hi=0.95).astype(np.float32)
        x0, y0 = int(rng.integers(0, W - sw)), int(rng.integers(0, H - sh))
        sprites.append((tex, x0, y0, int(rng.integers(-3, 4)), int(rng.integers(-2, 3))))
    out = np.empty((T, H, W, 3), np.float32)
    for t in range(T):
        out[t] = np.roll(bg, (vy * t, vx * t), axis=(0, 1))
        for tex, x0, y0, sx, sy in sprites:
            sh, sw = tex.shape[:2]
            x = (x0 + sx * t) % (W - sw)
            y = (y0 + sy * t) % (H - sh)
            out[t, y:y + sh, x:x + sw] = tex
    mask = _ellipse_tube(W, H, T, hole_frac, rng)
    return Clip(name or f"fast_{W}x{H}x{T}", out, mask, levels=0, use_texture=True,
                meta={"seed": seed, "hole_frac": hole_frac})


def serve_sizes(n=200, seed=BASE_SEED + 5):
    """Request sizes of the serving workload: W ~ logU[320, 1280], H ~
    logU[240, 720], frames ~ logU[30, 120] (even), hole fraction ~ U[3%, 10%]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        W = int(round(math.exp(rng.uniform(math.log(320), math.log(1280))) / 2)) * 2
        H = int(round(math.exp(rng.uniform(math.log(240), math.log(720))) / 2)) * 2
        T = int(round(math.exp(rng.uniform(math.log(30), math.log(120))) / 2)) * 2
        out.append((W, H, T, float(rng.uniform(0.03, 0.10))))
    return out


def batch_sizes(n=48, seed=BASE_SEED + 4):
    """Clip sizes for the batched workload: W ~ logU[160,640], H ~ logU[120,480],
    frames ~ logU[20,80], independently drawn and rounded to even sizes, plus a
    hole fraction ~ U[3%,12%] per clip."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        W = int(round(math.exp(rng.uniform(math.log(160), math.log(640))) / 2)) * 2
        H = int(round(math.exp(rng.uniform(math.log(120), math.log(480))) / 2)) * 2
        T = int(round(math.exp(rng.uniform(math.log(20), math.log(80))) / 2)) * 2
        out.append((W, H, T, float(rng.uniform(0.03, 0.12))))
    return out
