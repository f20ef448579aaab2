"""Pins for the patch distances of the oracle: Eq. 2 (colour), Eq. 7b (with
lambda-weighted texture channels) and Eq. 11 (partial distance), each against
closed forms and special cases, plus the expectation identity of Appendix B."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _two_regions(a, b, C=3, W=20, H=9, T=9):
    """x = a on the left half (x < 10), b on the right half."""
    x = np.full((T, H, W, C), a, np.float32)
    x[:, :, 10:, :] = b
    return x


@pytest.mark.parametrize("fp64", [False, True])
def test_self_distance_zero(fp64):
    rng = np.random.default_rng(0)
    x = rng.random((9, 9, 9, 5), dtype=np.float32)
    assert O.dist(x, (4, 4, 4), (4, 4, 4), fp64=fp64) == 0.0


@pytest.mark.parametrize("C", [1, 3, 5])
def test_constant_patches_closed_form(C):
    # target patch entirely in region a, source entirely in region b:
    # d^2 = (1/125) * 125 * C (a - b)^2 = C (a - b)^2
    a, b = 0.25, 0.75
    x = _two_regions(a, b, C)
    want = C * (a - b) ** 2
    assert O.dist(x, (4, 4, 4), (15, 4, 4), fp64=True) == pytest.approx(want, rel=1e-12)
    assert O.dist(x, (4, 4, 4), (15, 4, 4)) == pytest.approx(want, rel=1e-6)


def test_ramp_shift_closed_form():
    # u = alpha * x in every channel; a shift of s voxels in x changes every
    # term by alpha*s: d^2 = C (alpha s)^2, for any shift direction in y/t: 0.
    W, H, T, C = 40, 9, 9, 3
    alpha = 0.01
    xs = np.arange(W, dtype=np.float32) * np.float32(alpha)
    x = np.broadcast_to(xs[None, None, :, None], (T, H, W, C)).copy()
    for s in [1, 3, 7, -5]:
        want = C * (alpha * s) ** 2
        got = O.dist(x, (20, 4, 4), (20 + s, 4, 4), fp64=True)
        assert got == pytest.approx(want, rel=1e-5)
    assert O.dist(x, (20, 4, 4), (20, 2, 6), fp64=True) == 0.0


def test_border_target_divides_by_125():
    # a target at the corner keeps only its 3x3x3 in-volume offsets, and Eq. 2
    # still divides by N = 125: d^2 = 27 C (a-b)^2 / 125
    a, b, C = 0.25, 0.625, 3
    x = _two_regions(a, b, C, W=20, H=9, T=9)
    want = 27 * C * (a - b) ** 2 / 125.0
    assert O.dist(x, (0, 0, 0), (15, 4, 4), fp64=True) == pytest.approx(want, rel=1e-12)
    # on an edge (y = 0 only): 5 * 3 * 5 = 75 offsets
    want = 75 * C * (a - b) ** 2 / 125.0
    assert O.dist(x, (4, 0, 4), (15, 4, 4), fp64=True) == pytest.approx(want, rel=1e-12)


def test_source_outside_is_infinite():
    x = np.zeros((9, 9, 9, 3), np.float32)
    assert O.dist(x, (4, 4, 4), (1, 4, 4)) == math.inf
    assert O.dist(x, (4, 4, 4), (4, 4, 7)) == math.inf


def test_lambda_weights_texture_channels():
    # Eq. 7b: d^2 = (1/N) sum (|du|^2 + lambda |dT|^2). With identical colours
    # and texture features differing by c in T_x only, d^2 = lambda c^2.
    lam = 50.0
    W, H, T = 20, 9, 9
    rgb = np.full((T, H, W, 3), 0.5, np.float32)
    Tf = np.zeros((T, H, W, 2), np.float64)
    Tf[:, :, 10:, 0] = 0.03
    s = O.sqrt_lambda(lam)
    x = np.concatenate([rgb, (s * Tf).astype(np.float32)], axis=-1)
    got = O.dist(x, (4, 4, 4), (15, 4, 4), fp64=True)
    assert got == pytest.approx(lam * 0.03 ** 2, rel=1e-6)
    # and a pure colour difference is not weighted
    rgb2 = rgb.copy()
    rgb2[:, :, 10:, 1] = 0.7
    x2 = np.concatenate([rgb2, np.zeros((T, H, W, 2), np.float32)], axis=-1)
    assert O.dist(x2, (4, 4, 4), (15, 4, 4), fp64=True) == pytest.approx(0.2 ** 2, rel=1e-6)


def test_partial_distance_eq11():
    # Eq. 11: voxels of the current occlusion H' are left out and the sum is
    # divided by |N'_p|. Differences planted only on excluded voxels vanish.
    W, H, T, C = 20, 9, 9, 3
    x = np.full((T, H, W, C), 0.5, np.float32)
    excl = np.zeros((T, H, W), np.uint8)
    excl[3:6, 3:6, 3:6] = 1          # 27 voxels of the target patch of (4,4,4)
    x[3:6, 3:6, 3:6, :] = 0.875      # they differ from the source patch
    assert O.dist(x, (4, 4, 4), (15, 4, 4), excl=excl, fp64=True) == 0.0
    full = O.dist(x, (4, 4, 4), (15, 4, 4), fp64=True)
    assert full == pytest.approx(27 * C * 0.375 ** 2 / 125.0, rel=1e-12)
    # constant difference d on the kept voxels: mean over |N'_p| is C d^2
    x2 = np.full((T, H, W, C), 0.5, np.float32)
    x2[:, :, 10:, :] = 0.8
    assert O.dist(x2, (4, 4, 4), (15, 4, 4), excl=excl, fp64=True) == pytest.approx(
        C * 0.3 ** 2, rel=1e-6)
    # a patch whose every voxel is excluded has no distance
    excl_all = np.zeros((T, H, W), np.uint8)
    excl_all[2:7, 2:7, 2:7] = 1
    assert O.dist(x2, (4, 4, 4), (15, 4, 4), excl=excl_all) == math.inf


def test_fp32_close_to_fp64():
    rng = np.random.default_rng(1)
    x = rng.random((12, 12, 30, 5), dtype=np.float32)
    for _ in range(50):
        p = tuple(int(v) for v in (rng.integers(0, 30), rng.integers(0, 12), rng.integers(0, 12)))
        s = tuple(int(v) for v in (rng.integers(2, 28), rng.integers(2, 10), rng.integers(2, 10)))
        d32 = O.dist(x, p, s)
        d64 = O.dist(x, p, s, fp64=True)
        # 625 terms: |error| <= 625 * 2^-24 * sum, plus the final division
        assert abs(d32 - d64) <= 626 * 2 ** -24 * d64 + 1e-12


def test_symmetry_interior():
    rng = np.random.default_rng(2)
    x = rng.random((12, 12, 30, 3), dtype=np.float32)
    for p, s in [((5, 5, 5), (20, 6, 7)), ((3, 2, 2), (25, 9, 9))]:
        assert O.dist(x, p, s, fp64=True) == pytest.approx(O.dist(x, s, p, fp64=True), rel=1e-12)


def test_appendix_b_expectation_identity():
    # Appendix B: for i.i.d. patches W, V and the constant patch Z = mu,
    # E||W - V||^2 = 2 E||W - Z||^2. Checked with the oracle's comparator on
    # Gaussian patches (std 5, as in Table 2), 1-channel.
    rng = np.random.default_rng(5)
    W_, H_, T_ = 15, 5, 5
    n = 400
    dv, dz = [], []
    for _ in range(n):
        x = np.zeros((T_, H_, W_, 1), np.float32)
        x[:, :, 0:5, 0] = rng.normal(0.0, 5.0, (T_, H_, 5))     # W
        x[:, :, 5:10, 0] = rng.normal(0.0, 5.0, (T_, H_, 5))    # V
        dv.append(O.dist(x, (2, 2, 2), (7, 2, 2), fp64=True))
        dz.append(O.dist(x, (2, 2, 2), (12, 2, 2), fp64=True))   # Z = 0 = mu
    ratio = np.mean(dv) / np.mean(dz)
    assert ratio == pytest.approx(2.0, rel=0.03)
    assert np.mean(dz) == pytest.approx(25.0, rel=0.03)
