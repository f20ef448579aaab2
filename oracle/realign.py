"""Oracle for the affine realignment of Sec. 3.4 (Algorithm 2: AlignVideo) and
the final UnwarpVideo step of Algorithm 4.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU legs, never by the library. Plain FP64 numpy; loops only over
frames, pyramid levels and iterations.

The paper estimates "a dominant, affine motion between each pair of
successive frames" with the robust method of Odobez and Bouthemy and gives no
further detail. The reading fixed here (every choice is listed in the design
notes):

- motion model: a point p = (x, y) of frame n lies at A(p) = p + w(p) in
  frame n+1, w(p) = (a0 + a1 x + a2 y, a3 + a4 x + a5 y), pixel centres at
  integer coordinates;
- data term: grey-level constancy, I = (R + G + B) / 3, residual
  r(p) = I_{n+1}(A(p)) - I_n(p) with bilinear sampling; pixels occluded in
  frame n, samples outside frame n+1 and samples that touch an occluded pixel
  of frame n+1 (a neighbour with non-zero bilinear weight) take no part;
- robust fit: Gauss-Newton on the 6 parameters with iteratively reweighted
  least squares, Tukey's biweight with c = 4.6851 sigma, sigma^2 the weighted
  residual variance of the previous iteration (floor 1e-4), plain least
  squares in the very first iteration;
- multiresolution: 2x2 mean pyramid of the known pixels (sizes rounded up,
  occlusion by OR) down to a smallest side of at least 16, a fixed number of
  iterations per level, coarse to fine with the exact change of pixel
  coordinates X = 2x + 1/2;
- Algorithm 2: reference frame N_m = floor(N_f / 2) counted from 1 (index
  max(0, T // 2 - 1) from 0); theta_{n,N_m} is the product of the successive
  motions towards N_m (inverses after it); the aligned frame n samples u_n
  bilinearly at A_{n,N_m}^{-1}(q) for every pixel q of the reference grid;
  the occlusion is realigned with it, and a sample that falls outside frame n
  or touches an occluded pixel is occluded in the aligned video;
- UnwarpVideo: each originally occluded pixel y of frame n takes the aligned
  result at A_{n,N_m}(y) (bilinear, clamped to the frame); known pixels are
  kept.
"""
from __future__ import annotations

import math

import numpy as np

TUKEY_C = 4.6851
SIGMA_FLOOR = 1e-4


# --------------------------------------------------------------------------
# affine maps as 2x3 matrices [[m00, m01, m02], [m10, m11, m12]]
# --------------------------------------------------------------------------
def theta_to_matrix(a):
    """(a0..a5) -> the 2x3 matrix of p -> p + w(p)."""
    a = np.asarray(a, np.float64)
    return np.array([[1.0 + a[1], a[2], a[0]], [a[4], 1.0 + a[5], a[3]]])


def matrix_to_theta(m):
    return np.array([m[0, 2], m[0, 0] - 1.0, m[0, 1], m[1, 2], m[1, 0], m[1, 1] - 1.0])


def compose(m2, m1):
    """The map p -> m2(m1(p))."""
    return np.array([
        [m2[0, 0] * m1[0, 0] + m2[0, 1] * m1[1, 0], m2[0, 0] * m1[0, 1] + m2[0, 1] * m1[1, 1],
         m2[0, 0] * m1[0, 2] + m2[0, 1] * m1[1, 2] + m2[0, 2]],
        [m2[1, 0] * m1[0, 0] + m2[1, 1] * m1[1, 0], m2[1, 0] * m1[0, 1] + m2[1, 1] * m1[1, 1],
         m2[1, 0] * m1[0, 2] + m2[1, 1] * m1[1, 2] + m2[1, 2]]])


def invert(m):
    """Closed-form inverse of the affine map, in a fixed operation order (the
    library's host code evaluates the same expressions)."""
    det = m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0]
    i00 = m[1, 1] / det
    i01 = -m[0, 1] / det
    i10 = -m[1, 0] / det
    i11 = m[0, 0] / det
    i02 = -(i00 * m[0, 2] + i01 * m[1, 2])
    i12 = -(i10 * m[0, 2] + i11 * m[1, 2])
    return np.array([[i00, i01, i02], [i10, i11, i12]])


def apply(m, x, y):
    """m(x, y), evaluated as (m0 * x + m1 * y) + m2."""
    return m[0, 0] * x + m[0, 1] * y + m[0, 2], m[1, 0] * x + m[1, 1] * y + m[1, 2]


# --------------------------------------------------------------------------
# images
# --------------------------------------------------------------------------
def grey(rgb):
    rgb = np.asarray(rgb, np.float64)
    return (rgb[..., 0] + rgb[..., 1] + rgb[..., 2]) / 3.0


def gradients(I):
    """Central differences, one-sided on the frame border (0 for a side of 1)."""
    H, W = I.shape
    gx = np.zeros_like(I)
    gy = np.zeros_like(I)
    if W > 1:
        gx[:, 1:-1] = (I[:, 2:] - I[:, :-2]) / 2.0
        gx[:, 0] = I[:, 1] - I[:, 0]
        gx[:, -1] = I[:, -1] - I[:, -2]
    if H > 1:
        gy[1:-1] = (I[2:] - I[:-2]) / 2.0
        gy[0] = I[1] - I[0]
        gy[-1] = I[-1] - I[-2]
    return gx, gy


def downsample(I, occ):
    """2x2 mean of the known children (sizes rounded up); a coarse pixel is
    occluded when any child is."""
    H, W = I.shape
    h, w = (H + 1) // 2, (W + 1) // 2
    s = np.zeros((h, w))
    n = np.zeros((h, w))
    o = np.zeros((h, w), np.uint8)
    for dy in (0, 1):
        for dx in (0, 1):
            sub = I[dy::2, dx::2]
            so = occ[dy::2, dx::2]
            hh, ww = sub.shape
            known = so == 0
            s[:hh, :ww] += np.where(known, sub, 0.0)
            n[:hh, :ww] += known
            o[:hh, :ww] |= so
    return np.where(n > 0, s / np.maximum(n, 1), 0.0), o


def pyramid_levels(W, H):
    L = 1
    while L < 6 and (min(W, H) + (1 << L) - 1) // (1 << L) >= 16:
        L += 1
    return L


def sample_bilinear(img, qx, qy):
    """Bilinear samples at (qx, qy) (inside [0, W-1] x [0, H-1]); also the
    indices and which of the four neighbours have a non-zero weight."""
    H, W = img.shape[:2]
    x0 = np.floor(qx).astype(np.int64)
    y0 = np.floor(qy).astype(np.int64)
    fx = qx - x0
    fy = qy - y0
    x0 = np.clip(x0, 0, W - 1)
    y0 = np.clip(y0, 0, H - 1)
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    if img.ndim == 3:
        fxe, fye = fx[..., None], fy[..., None]
    else:
        fxe, fye = fx, fy
    v = ((1.0 - fye) * ((1.0 - fxe) * img[y0, x0] + fxe * img[y0, x1])
         + fye * ((1.0 - fxe) * img[y1, x0] + fxe * img[y1, x1]))
    return v, (x0, y0, x1, y1, fx > 0, fy > 0)


def touches(occ, nb):
    """Whether a bilinear sample reads an occluded pixel (with non-zero weight)."""
    x0, y0, x1, y1, ux, uy = nb
    return ((occ[y0, x0] != 0) | (ux & (occ[y0, x1] != 0)) | (uy & (occ[y1, x0] != 0))
            | (ux & uy & (occ[y1, x1] != 0)))


# --------------------------------------------------------------------------
# EstimateAffineMotion
# --------------------------------------------------------------------------
def tukey(r, c):
    if not math.isfinite(c):
        return np.ones_like(r)
    u = r / c
    return np.where(np.abs(r) < c, (1.0 - u * u) ** 2, 0.0)


def gauss_newton_step(I1, o1, I2, o2, gx2, gy2, theta, c):
    """One IRLS Gauss-Newton step at one level. Returns (delta, sum w r^2,
    sum w); delta is 0 when the system is empty or singular."""
    H, W = I1.shape
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    m = theta_to_matrix(theta)
    qx, qy = apply(m, xx, yy)
    inside = (qx >= 0) & (qx <= W - 1) & (qy >= 0) & (qy <= H - 1) & (o1 == 0)
    qxc = np.where(inside, qx, 0.0)
    qyc = np.where(inside, qy, 0.0)
    v, nb = sample_bilinear(I2, qxc, qyc)
    ok = inside & ~touches(o2, nb)
    gx, _ = sample_bilinear(gx2, qxc, qyc)
    gy, _ = sample_bilinear(gy2, qxc, qyc)
    r = v - I1
    w = np.where(ok, tukey(r, c), 0.0)
    J = np.stack([gx, gx * xx, gx * yy, gy, gy * xx, gy * yy], -1)
    Jw = J * w[..., None]
    A = np.einsum("hwi,hwj->ij", Jw, J)
    b = np.einsum("hwi,hw->i", Jw, r)
    sw = float(w.sum())
    swr2 = float((w * r * r).sum())
    delta = np.zeros(6)
    if sw > 0.0:
        ridge = 1e-9 * (np.trace(A) / 6.0) + 1e-30
        try:
            delta = np.linalg.solve(A + ridge * np.eye(6), -b)
        except np.linalg.LinAlgError:
            delta = np.zeros(6)
        if not np.all(np.isfinite(delta)):
            delta = np.zeros(6)
    return delta, swr2, sw


def estimate_pair(I1, o1, I2, o2, levels=None, iters=10):
    """theta_{n,n+1}: the dominant affine motion from frame n (I1, occlusion
    o1) to frame n+1 (I2, o2)."""
    H, W = I1.shape
    if levels is None:
        levels = pyramid_levels(W, H)
    p1, p2 = [(np.asarray(I1, np.float64), np.asarray(o1, np.uint8))], \
        [(np.asarray(I2, np.float64), np.asarray(o2, np.uint8))]
    for _ in range(levels - 1):
        p1.append(downsample(*p1[-1]))
        p2.append(downsample(*p2[-1]))
    theta = np.zeros(6)
    c = math.inf
    for lev in range(levels - 1, -1, -1):
        A1, B1 = p1[lev]
        A2, B2 = p2[lev]
        gx2, gy2 = gradients(A2)
        for _ in range(iters):
            delta, swr2, sw = gauss_newton_step(A1, B1, A2, B2, gx2, gy2, theta, c)
            theta = theta + delta
            if sw > 0.0:
                c = TUKEY_C * max(math.sqrt(swr2 / sw), SIGMA_FLOOR)
        if lev > 0:
            theta = theta.copy()
            theta[0] = 2.0 * theta[0] - 0.5 * (theta[1] + theta[2])
            theta[3] = 2.0 * theta[3] - 0.5 * (theta[4] + theta[5])
    return theta


def estimate(rgb, mask, levels=None, iters=10):
    """Algorithm 2, first loop: theta_{n,n+1} for n = 0 .. T-2, as [T-1][6]."""
    I = grey(rgb)
    mask = np.asarray(mask, np.uint8)
    T = I.shape[0]
    return np.array([estimate_pair(I[n], mask[n], I[n + 1], mask[n + 1], levels, iters)
                     for n in range(T - 1)]).reshape(-1, 6)


# --------------------------------------------------------------------------
# AlignVideo / UnwarpVideo
# --------------------------------------------------------------------------
def reference_frame(T):
    return max(0, T // 2 - 1)


def to_reference(theta_pairs, T):
    """theta_{n,N_m} for every frame n, as 2x3 matrices [T][2][3]."""
    r = reference_frame(T)
    mats = [theta_to_matrix(t) for t in np.asarray(theta_pairs).reshape(-1, 6)]
    out = [None] * T
    out[r] = theta_to_matrix(np.zeros(6))
    for n in range(r - 1, -1, -1):          # A_{n,r} = A_{n+1,r} o A_{n,n+1}
        out[n] = compose(out[n + 1], mats[n])
    for n in range(r + 1, T):               # A_{n,r} = A_{n-1,r} o A_{n-1,n}^-1
        out[n] = compose(out[n - 1], invert(mats[n - 1]))
    return np.array(out)


def align(rgb, mask, to_ref):
    """The aligned video and occlusion: frame n sampled at A_{n,N_m}^{-1}(q)."""
    rgb = np.asarray(rgb, np.float64)
    mask = np.asarray(mask, np.uint8)
    T, H, W = mask.shape
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.zeros_like(rgb)
    occ = np.ones_like(mask)
    for n in range(T):
        px, py = apply(invert(to_ref[n]), xx, yy)
        inside = (px >= 0) & (px <= W - 1) & (py >= 0) & (py <= H - 1)
        v, nb = sample_bilinear(rgb[n], np.where(inside, px, 0.0), np.where(inside, py, 0.0))
        out[n] = np.where(inside[..., None], v, 0.0)
        occ[n] = (~inside | touches(mask[n], nb)).astype(np.uint8)
    return out, occ


def unwarp(rgb, mask, aligned_result, to_ref):
    """UnwarpVideo: originally occluded pixels take the aligned result at
    A_{n,N_m}(y) (bilinear, clamped to the frame); known pixels are kept."""
    out = np.array(rgb, np.float64)
    mask = np.asarray(mask, np.uint8)
    aligned_result = np.asarray(aligned_result, np.float64)
    T, H, W = mask.shape
    for n in range(T):
        ys, xs = np.nonzero(mask[n])
        if len(ys) == 0:
            continue
        qx, qy = apply(to_ref[n], xs.astype(np.float64), ys.astype(np.float64))
        qx = np.clip(qx, 0.0, W - 1.0)
        qy = np.clip(qy, 0.0, H - 1.0)
        v, _ = sample_bilinear(aligned_result[n], qx, qy)
        out[n, ys, xs] = v
    return out
