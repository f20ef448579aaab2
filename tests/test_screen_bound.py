"""The error bound behind FP16 screening, checked in FP64 on the CPU.

For FP32 channel values a, b with |a|, |b| <= M_c in channel c and their
FP16 roundings a', b', every entry of e = (a' - b') - (a - b) is at most
delta_c = 2^-10 M_c + 2^-24, hence |x'| - |x| <= |e| <= sqrt(k D) with
D = sum_c delta_c^2 over the k voxels of a patch. The screening rejects a
candidate only when sqrt(S') - sqrt(k D) proves S large enough; these tests
check the inequality on random, adversarial (rounding midpoints, FP16
subnormals, the range limit) and structured inputs."""
import numpy as np


def _delta(M):
    return np.float64(2.0 ** -10) * M + np.float64(2.0 ** -24)


def _check(a, b):
    """a, b: [k, C] float32 values. Returns the slack of the bound (>= 0)."""
    M = np.maximum(np.abs(a).max(0), np.abs(b).max(0)).astype(np.float64)
    x = a.astype(np.float64) - b.astype(np.float64)
    xh = a.astype(np.float16).astype(np.float64) - b.astype(np.float16).astype(np.float64)
    e = xh - x
    assert (np.abs(e) <= _delta(M)[None, :]).all()
    k = a.shape[0]
    D = float((_delta(M) ** 2).sum())
    lower = np.sqrt((xh ** 2).sum()) - np.sqrt(k * D)
    return np.sqrt((x ** 2).sum()) - lower


def test_random_patches():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        M = rng.choice([1.0, 3.5, 0.01, 200.0])
        a = (rng.random((125, 5)) * 2 - 1).astype(np.float32) * np.float32(M)
        b = a + (rng.standard_normal((125, 5)) * rng.choice([1e-4, 1e-2, 1.0]) * M).astype(np.float32)
        b = np.clip(b, -M, M).astype(np.float32)
        assert _check(a, b) >= 0


def test_rounding_midpoints():
    # values halfway between FP16 neighbours: the largest rounding errors
    rng = np.random.default_rng(2)
    base = rng.random((125, 5)).astype(np.float16).astype(np.float32)
    ulp = (np.spacing(base.astype(np.float16)).astype(np.float32))
    a = (base + ulp / 2).astype(np.float32)
    b = (base - ulp / 2 + ulp / 4).astype(np.float32)
    assert _check(a, b) >= 0
    assert _check(a, base) >= 0


def test_subnormal_and_range_limit():
    rng = np.random.default_rng(3)
    tiny = (rng.random((125, 5)) * 2 ** -15).astype(np.float32)       # FP16 subnormals
    assert _check(tiny, np.zeros_like(tiny)) >= 0
    assert _check(tiny, (tiny * 0.5).astype(np.float32)) >= 0
    big = (rng.random((125, 5)) * 65504.0).astype(np.float32)         # up to the FP16 maximum
    assert _check(big, (big * 0.999).astype(np.float32)) >= 0


def test_identical_patches_pass():
    # S = 0 (a perfect match): the lower bound must not exceed 0
    rng = np.random.default_rng(4)
    a = rng.random((125, 5)).astype(np.float32)
    assert _check(a, a.copy()) >= 0
    x16 = a.astype(np.float16).astype(np.float64)
    assert np.sqrt(((x16 - x16) ** 2).sum()) == 0.0


def test_partial_sums():
    # the bound on the first j slices (k = 25 j voxels) lower-bounds the full sum
    rng = np.random.default_rng(5)
    for _ in range(500):
        a = rng.random((125, 5)).astype(np.float32)
        b = rng.random((125, 5)).astype(np.float32)
        M = np.maximum(np.abs(a).max(0), np.abs(b).max(0)).astype(np.float64)
        D = float((_delta(M) ** 2).sum())
        x = a.astype(np.float64) - b.astype(np.float64)
        xh = a.astype(np.float16).astype(np.float64) - b.astype(np.float16).astype(np.float64)
        S_full = (x ** 2).sum()
        for j in range(1, 6):
            k = 25 * j
            lower = np.sqrt((xh[:k] ** 2).sum()) - np.sqrt(k * D)
            assert np.sqrt(S_full) >= lower
