"""CPU oracle for "Video Inpainting of Complex Scenes" (Newson et al.,
arXiv:1503.05528): Python side.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The CUDA library never calls it and shares no code with it.

The per-voxel arithmetic lives in ``vi_oracle.c`` (plain C loops, compiled
with gcc ``-O2 -ffp-contract=off``); this file loads it with ctypes and
strings the steps together in the order of Algorithm 4 (the complete method)
and Algorithm 3 (onion-peel initialisation). Arrays are numpy, C-contiguous,
shaped ``[T][H][W]`` (masks, distances) and ``[T][H][W][C]`` (channels) or
``[T][H][W][3]`` (shift maps, int32 dx, dy, dt).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vi_oracle.c")
_SO = os.path.join(_HERE, "_build", "libvi_oracle.so")

# Random-draw purposes (the 4 high bits of the Philox tag word).
PURPOSE_INIT = 1        # phi^L <- Random (Algorithm 4)
PURPOSE_SEARCH = 2      # random search of the main loop (Eq. 3)
PURPOSE_UPSAMPLE = 3    # redraw of an upsampled shift that left D~
PURPOSE_ONION = 4       # random search during the initialisation (Algorithm 3)


def tag(purpose, level, call=0, k=0):
    """Philox counter word 1: purpose (4 bits), level (4), call (16), k (8)."""
    return ((purpose & 0xF) << 28) | ((level & 0xF) << 24) | ((call & 0xFFFF) << 8) | (k & 0xFF)


def build(force=False):
    """Compile the oracle with gcc (a test-only C library)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


class _OptU8:
    """ctypes converter accepting a uint8 array or None (NULL)."""

    @classmethod
    def from_param(cls, obj):
        if obj is None:
            return None
        assert obj.dtype == np.uint8 and obj.flags.c_contiguous
        return obj.ctypes.data_as(C.c_void_p)


def _declare(L):
    i, u32, d = C.c_int, C.c_uint32, C.c_double
    L.vio_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.vio_unit_symmetric.argtypes = [u32]
    L.vio_unit_symmetric.restype = d
    L.vio_uniform_index.argtypes = [u32, u32]
    L.vio_uniform_index.restype = u32
    dist_args = [_f32p, i, i, i, i, i, i, i, i, i, i, _OptU8]
    L.vio_dist_f32.argtypes = dist_args
    L.vio_dist_f32.restype = C.c_float
    L.vio_dist_f64.argtypes = dist_args
    L.vio_dist_f64.restype = d
    L.vio_dilate5.argtypes = [_u8p, i, i, i, _u8p]
    L.vio_masks.argtypes = [_u8p, i, i, i, _u8p, _u8p]
    L.vio_erode3.argtypes = [_u8p, i, i, i, _u8p]
    L.vio_texture_features.argtypes = [_f32p, _u8p, i, i, i, i, _f64p]
    L.vio_subsample_features.argtypes = [_f64p, i, i, i, i, i, i, _f64p]
    L.vio_downsample.argtypes = [_f32p, _u8p, i, i, i, i, _f32p, _u8p]
    L.vio_init_nnf.argtypes = [_u8p, _u8p, i, i, i, u32, u32, u32, u32, _i32p]
    L.vio_init_nnf.restype = i
    L.vio_upsample_nnf.argtypes = [_i32p, i, i, _u8p, _u8p, i, i, i, u32, u32, u32, u32, _i32p]
    L.vio_upsample_nnf.restype = i
    L.vio_subsample_features_t.argtypes = [_f64p, i, i, i, i, i, i, i, i, _f64p]
    L.vio_downsample_t.argtypes = [_f32p, _u8p, i, i, i, i, i, _f32p, _u8p]
    L.vio_upsample_nnf_t.argtypes = [_i32p, i, i, i, _u8p, _u8p, i, i, i, i, u32, u32, u32, u32, _i32p]
    L.vio_upsample_nnf_t.restype = i
    L.vio_ann.argtypes = [_f32p, i, i, i, i, _u8p, _u8p, _OptU8, _i32p, _f32p, i, i, i, d,
                          u32, u32, u32, u32]
    L.vio_ann.restype = C.c_longlong
    L.vio_ann2.argtypes = [_f32p, i, i, i, i, _u8p, _u8p, _OptU8, _i32p, _f32p, i, i, i, d,
                           u32, u32, u32, u32, i, i]
    L.vio_ann2.restype = C.c_longlong
    L.vio_ann2_f64.argtypes = [_f32p, i, i, i, i, _u8p, _u8p, _OptU8, _i32p, _f64p, i, i, i, d,
                               u32, u32, u32, u32, i, i]
    L.vio_ann2_f64.restype = C.c_longlong
    L.vio_rescore.argtypes = [_f32p, i, i, i, i, _u8p, _u8p, _OptU8, _i32p, _f32p]
    L.vio_rescore.restype = C.c_longlong
    L.vio_ann_iteration.argtypes = [_f32p, i, i, i, i, _u8p, _OptU8, _u8p, _OptU8, _i32p, _f32p, i, i, d,
                                    u32, u32, u32, u32, i, i]
    L.vio_ann_iteration.restype = C.c_longlong
    L.vio_bruteforce_nn.argtypes = [_f32p, i, i, i, i, _u8p, _u8p, _OptU8, _i32p, _f32p]
    L.vio_vote.argtypes = [_f32p, _f32p, i, i, i, i, _u8p, _u8p, _i32p, _f32p, i, i, _OptU8]
    L.vio_vote.restype = d
    L.vio_vote_f64.argtypes = [_f32p, _f32p, i, i, i, i, _u8p, _u8p, _i32p, _f64p, i, i, _OptU8]
    L.vio_vote_f64.restype = d
    L.vio_final_f64.argtypes = [_f32p, _f32p, i, i, i, i, _u8p, _i32p, _f64p]
    L.vio_final.argtypes = [_f32p, _f32p, i, i, i, i, _u8p, _i32p, _f32p]
    L.vio_energy.argtypes = [_f32p, i, i, i, i, _u8p, _u8p, _i32p, _f64p]


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dims(mask):
    T, H, W = mask.shape
    return W, H, T


# --------------------------------------------------------------------------
# Step wrappers (one C routine each)
# --------------------------------------------------------------------------

def philox4x32_10(counter, key):
    out = np.zeros(4, np.uint32)
    lib().vio_philox4x32_10(_c(counter, np.uint32), _c(key, np.uint32), out)
    return out


def unit_symmetric(w):
    return lib().vio_unit_symmetric(int(w))


def uniform_index(w, n):
    return lib().vio_uniform_index(int(w), int(n))


def dist(x, p, s, excl=None, fp64=False):
    """Squared patch distance d^2(W_p, W_s) (Eq. 2 / 7b; Eq. 11 with ``excl``).
    ``x`` is [T][H][W][C] float32; p and s are (x, y, t)."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    fn = lib().vio_dist_f64 if fp64 else lib().vio_dist_f32
    return fn(x.reshape(-1), W, H, T, Cn, p[0], p[1], p[2], s[0], s[1], s[2],
              None if excl is None else _c(excl, np.uint8).reshape(-1))


def dilate5(m):
    m = _c(m, np.uint8)
    W, H, T = _dims(m)
    out = np.zeros_like(m)
    lib().vio_dilate5(m.reshape(-1), W, H, T, out.reshape(-1))
    return out


def erode3(m):
    m = _c(m, np.uint8)
    W, H, T = _dims(m)
    out = np.zeros_like(m)
    lib().vio_erode3(m.reshape(-1), W, H, T, out.reshape(-1))
    return out


def masks(hole):
    """(H~, D~) of Sec. 2 for an occlusion mask."""
    hole = _c(hole, np.uint8)
    W, H, T = _dims(hole)
    ht = np.zeros_like(hole)
    dt = np.zeros_like(hole)
    lib().vio_masks(hole.reshape(-1), W, H, T, ht.reshape(-1), dt.reshape(-1))
    return ht, dt


def texture_features(rgb, hole, nu_side):
    """Eq. 7 at full resolution: float64 [T][H][W][2]."""
    rgb = _c(rgb, np.float32)
    hole = _c(hole, np.uint8)
    W, H, T = _dims(hole)
    out = np.zeros((T, H, W, 2), np.float64)
    lib().vio_texture_features(rgb.reshape(-1), hole.reshape(-1), W, H, T, int(nu_side),
                               out.reshape(-1))
    return out


def subsample_features(T0, level, Wl, Hl, Tl=None, tsub=False):
    """Eq. 8: T^l(x, y, t) = T(2^l x, 2^l y, t); with tsub T(2^l x, 2^l y, 2^l t)."""
    T0 = _c(T0, np.float64)
    T, H0, W0, _ = T0.shape
    Tl = T if Tl is None else Tl
    out = np.zeros((Tl, Hl, Wl, 2), np.float64)
    lib().vio_subsample_features_t(T0.reshape(-1), W0, H0, T, int(level), Wl, Hl, Tl, 1 if tsub else 0,
                                   out.reshape(-1))
    return out


def downsample(x, hole, tsub=False):
    """One level of the colour / occlusion pyramids (2x2, or 2x2x2 with tsub)."""
    x = _c(x, np.float32)
    hole = _c(hole, np.uint8)
    T, Hf, Wf, Cn = x.shape
    Wc, Hc = (Wf + 1) // 2, (Hf + 1) // 2
    Tc = (T + 1) // 2 if tsub else T
    xc = np.zeros((Tc, Hc, Wc, Cn), np.float32)
    hc = np.zeros((Tc, Hc, Wc), np.uint8)
    lib().vio_downsample_t(x.reshape(-1), hole.reshape(-1), Wf, Hf, T, Cn, 1 if tsub else 0, xc.reshape(-1),
                           hc.reshape(-1))
    return xc, hc


def init_nnf(target, dtilde, key, tag_word, clip=0):
    target = _c(target, np.uint8)
    W, H, T = _dims(target)
    phi = np.zeros((T, H, W, 3), np.int32)
    rc = lib().vio_init_nnf(target.reshape(-1), _c(dtilde, np.uint8).reshape(-1), W, H, T,
                            key[0], key[1], tag_word, clip, phi.reshape(-1))
    if rc != 0:
        raise ValueError("no valid source patch (D~ is empty)")
    return phi


def upsample_nnf(phi_c, target_f, dtilde_f, key, tag_word, clip=0, tsub=False):
    phi_c = _c(phi_c, np.int32)
    Tc, Hc, Wc, _ = phi_c.shape
    target_f = _c(target_f, np.uint8)
    Wf, Hf, T = _dims(target_f)
    phi_f = np.zeros((T, Hf, Wf, 3), np.int32)
    rc = lib().vio_upsample_nnf_t(phi_c.reshape(-1), Wc, Hc, Tc, target_f.reshape(-1),
                                  _c(dtilde_f, np.uint8).reshape(-1), Wf, Hf, T, 1 if tsub else 0,
                                  key[0], key[1], tag_word, clip, phi_f.reshape(-1))
    if rc != 0:
        raise ValueError("no valid source patch (D~ is empty)")
    return phi_f


def ann(x, target, dtilde, phi, d2, n_pm=10, schedule="JAC", rmax=None, rho=0.5,
        key=(0, 0), tag_base=0, clip=0, excl=None, rs_mode=0, sub_sweeps=1):
    """Algorithm 1 in place on (phi, d2). Returns the number of distance
    evaluations. ``schedule``: "SEQ" (Algorithm 1 as printed) or "JAC".
    ``d2`` float32: FP32 distances in the canonical summation order (the
    GPU's); float64: distances and decisions in FP64 (the FP64 reference).
    ``rs_mode`` 0: one random candidate per k at radius r_max rho^k (Eq. 3);
    1: a candidate at every radius r_max rho^i >= 1 per k (the original
    PatchMatch search). ``sub_sweeps``: propagation sweeps before each random
    search."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    assert phi.dtype == np.int32 and phi.flags.c_contiguous
    assert d2.dtype in (np.float32, np.float64) and d2.flags.c_contiguous
    if rmax is None:
        rmax = max(W, H, T)
    sched = {"SEQ": 0, "JAC": 1}[schedule]
    assert rs_mode in (0, 1) and sub_sweeps >= 1
    fn = lib().vio_ann2_f64 if d2.dtype == np.float64 else lib().vio_ann2
    return fn(x.reshape(-1), W, H, T, Cn, _c(target, np.uint8).reshape(-1),
                          _c(dtilde, np.uint8).reshape(-1),
                          None if excl is None else _c(excl, np.uint8).reshape(-1),
                          phi.reshape(-1), d2.reshape(-1), int(n_pm), sched, int(rmax),
                          float(rho), key[0], key[1], int(tag_base), int(clip), int(rs_mode),
                          int(sub_sweeps))


def rescore(x, target, dtilde, phi, d2, excl=None):
    """The first step of ann (JAC): every target's distance to its current
    correspondent, in place in d2. Returns the evaluations."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    assert phi.dtype == np.int32 and phi.flags.c_contiguous
    assert d2.dtype == np.float32 and d2.flags.c_contiguous
    return lib().vio_rescore(x.reshape(-1), W, H, T, Cn, _c(target, np.uint8).reshape(-1),
                             _c(dtilde, np.uint8).reshape(-1),
                             None if excl is None else _c(excl, np.uint8).reshape(-1),
                             phi.reshape(-1), d2.reshape(-1))


def ann_iteration(x, target, dtilde, phi, d2, k, rmax=None, rho=0.5, key=(0, 0), tag_base=0, clip=0,
                  excl=None, rs_mode=0, sub_sweeps=1, own=None):
    """Iteration k of ann with the Jacobi schedule, in place, for the targets
    in own (None: all of target; target still says which neighbours hold a
    shift). rescore then ann_iteration for k = 1 .. n_pm is
    ann(schedule="JAC"). Returns the evaluations."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    assert phi.dtype == np.int32 and phi.flags.c_contiguous
    assert d2.dtype == np.float32 and d2.flags.c_contiguous
    if rmax is None:
        rmax = max(W, H, T)
    n = lib().vio_ann_iteration(x.reshape(-1), W, H, T, Cn, _c(target, np.uint8).reshape(-1),
                                None if own is None else _c(own, np.uint8).reshape(-1),
                                _c(dtilde, np.uint8).reshape(-1),
                                None if excl is None else _c(excl, np.uint8).reshape(-1),
                                phi.reshape(-1), d2.reshape(-1), int(k), int(rmax), float(rho), key[0], key[1],
                                int(tag_base), int(clip), int(rs_mode), int(sub_sweeps))
    if n < 0:
        raise MemoryError("vio_ann_iteration")
    return n


def bruteforce_nn(x, target, dtilde, excl=None):
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    phi = np.zeros((T, H, W, 3), np.int32)
    d2 = np.full((T, H, W), np.inf, np.float32)
    lib().vio_bruteforce_nn(x.reshape(-1), W, H, T, Cn, _c(target, np.uint8).reshape(-1),
                            _c(dtilde, np.uint8).reshape(-1),
                            None if excl is None else _c(excl, np.uint8).reshape(-1),
                            phi.reshape(-1), d2.reshape(-1))
    return phi, d2


def vote(x, vote_mask, allowed, phi, d2, weighted=True, n_diff=3, want_deferred=False):
    """Eq. 4/5 (Eq. 9, Eq. 12). Returns (x_new, change_sum[, deferred]).
    Weights and sums in FP64; d2 float32 or float64."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    out = np.empty_like(x)
    deferred = np.zeros((T, H, W), np.uint8) if want_deferred else None
    f64 = np.asarray(d2).dtype == np.float64
    fn = lib().vio_vote_f64 if f64 else lib().vio_vote
    ch = fn(x.reshape(-1), out.reshape(-1), W, H, T, Cn,
                        _c(vote_mask, np.uint8).reshape(-1), _c(allowed, np.uint8).reshape(-1),
                        _c(phi, np.int32).reshape(-1), _c(d2, np.float64 if f64 else np.float32).reshape(-1),
                        1 if weighted else 0, int(n_diff),
                        None if deferred is None else deferred.reshape(-1))
    if want_deferred:
        return out, ch, deferred
    return out, ch


def final(x, hole, phi, d2):
    """Eq. 6."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    out = np.empty_like(x)
    f64 = np.asarray(d2).dtype == np.float64
    fn = lib().vio_final_f64 if f64 else lib().vio_final
    fn(x.reshape(-1), out.reshape(-1), W, H, T, Cn, _c(hole, np.uint8).reshape(-1),
       _c(phi, np.int32).reshape(-1), _c(d2, np.float64 if f64 else np.float32).reshape(-1))
    return out


def energy(x, hole, htilde, phi):
    """Eq. 1 in FP64: (E_H, E_H~)."""
    x = _c(x, np.float32)
    T, H, W, Cn = x.shape
    out = np.zeros(2, np.float64)
    lib().vio_energy(x.reshape(-1), W, H, T, Cn, _c(hole, np.uint8).reshape(-1),
                     _c(htilde, np.uint8).reshape(-1), _c(phi, np.int32).reshape(-1), out)
    return float(out[0]), float(out[1])


# --------------------------------------------------------------------------
# The complete method (Algorithm 4, without the affine realignment of Alg. 2)
# --------------------------------------------------------------------------

@dataclass
class Params:
    """Parameters of Sec. 3.7."""

    lam: float = 50.0          # lambda, texture weight (Eq. 7b)
    n_pm: int = 10             # PatchMatch iterations per ANN search
    rho: float = 0.5           # radius reduction factor (Eq. 3)
    max_outer: int = 20        # iteration cap per level
    stop: float = 0.1 / 255.0  # threshold on e (Sec. 3.7, on [0, 1] colour)
    weighted: bool = True      # Eq. 4/5 weights (False: s = 1)
    seed: int = 1503
    clip: int = 0
    schedule: str = "JAC"      # "SEQ" (Algorithm 1 as printed) or "JAC"
    fixed_outer: object = None  # None, an int, or a list per level (coarsest first)
    rs_mode: int = 0           # 0: Eq. 3 (one radius per k); 1: every radius r_max rho^i >= 1
    sub_sweeps: int = 1        # propagation sweeps before each random search
    time_subsample: bool = False  # halve the frames at every pyramid level too (Sec. 3.6 option)
    fp64: bool = False         # distances, stored distances and decisions in FP64 (the reference
                               # the FP32 path's errors are stated against); the video stays FP32

    @property
    def d2_dtype(self):
        return np.float64 if self.fp64 else np.float32

    @property
    def key(self):
        return (self.seed & 0xFFFFFFFF, (self.seed >> 32) & 0xFFFFFFFF)


@dataclass
class Level:
    x: np.ndarray          # float32 [T][H][W][C]
    hole: np.ndarray       # uint8 [T][H][W]
    htilde: np.ndarray
    dtilde: np.ndarray
    phi: np.ndarray = None  # int32 [T][H][W][3]
    d2: np.ndarray = None   # float32 [T][H][W]
    stats: dict = field(default_factory=dict)

    @property
    def dims(self):
        T, H, W, _ = self.x.shape
        return W, H, T


def sqrt_lambda(lam):
    """sqrt(lambda) rounded once to float32: texture channels are stored
    pre-multiplied by it so that Eq. 7b is a plain SSD over 5 channels."""
    return float(np.float32(math.sqrt(lam)))


def build_pyramid(rgb, mask, levels, use_texture=True, lam=50.0, tsub=False):
    """ImagePyramid, TextureFeaturePyramid and OcclusionPyramid of Algorithm 4
    (level 0 = finest). Channels: R, G, B (+ sqrt(lambda) T_x, sqrt(lambda) T_y).
    Values on occluded voxels are unknown and set to 0. tsub: the temporal
    subsampling option (frames halved at every level too)."""
    rgb = _c(rgb, np.float32)
    mask = _c(mask, np.uint8)
    T0 = None
    if use_texture:
        T0 = texture_features(rgb, mask, 2 ** (levels - 1))
    s = sqrt_lambda(lam)
    out = []
    col, hole = rgb.copy(), mask.copy()
    for lv in range(levels):
        if lv > 0:
            col, hole = downsample(col, hole, tsub)
        T, H, W, _ = col.shape
        if use_texture:
            Tl = subsample_features(T0, lv, W, H, T, tsub)
            x = np.concatenate([col, (s * Tl).astype(np.float32)], axis=-1)
        else:
            x = col.copy()
        x[hole.astype(bool)] = 0.0
        ht, dt = masks(hole)
        out.append(Level(np.ascontiguousarray(x), hole, ht, dt))
    return out


def _rescore(lv, prm, excl=None, target=None):
    """Distances of the targets to their current correspondents (an ANN call
    with no PatchMatch iteration)."""
    return ann(lv.x, lv.htilde if target is None else target, lv.dtilde, lv.phi, lv.d2,
               n_pm=0, schedule=prm.schedule, rho=prm.rho, key=prm.key, excl=excl)


def onion_layer(lv, prm, level_index, n_layer, Hp):
    """One layer of Algorithm 3 on H' = Hp (uint8): dH' = H' minus its 3x3x3
    erosion; the ANN search (Algorithm 1, partial distance of Eq. 11, random
    draws tagged with the layer) for the patches that meet dH' and are centred
    outside H'; the vote of dH' with Eq. 12 from those patches only. Updates
    lv.x, lv.phi and lv.d2 in place and returns (new H', evaluations): the
    erosion of H' plus the layer voxels that no such patch covers."""
    eroded = erode3(Hp)
    layer = Hp & (1 - eroded)
    targets = dilate5(layer) & (1 - Hp)
    evals = ann(lv.x, targets, lv.dtilde, lv.phi, lv.d2, n_pm=prm.n_pm,
                schedule=prm.schedule, rho=prm.rho, key=prm.key,
                tag_base=tag(PURPOSE_ONION, level_index, n_layer), clip=prm.clip, excl=Hp,
                rs_mode=prm.rs_mode, sub_sweeps=prm.sub_sweeps)
    x_new, _, deferred = vote(lv.x, layer, targets, lv.phi, lv.d2, weighted=prm.weighted,
                              n_diff=0, want_deferred=True)
    lv.x = x_new
    return (eroded | (layer & deferred)).astype(np.uint8), evals


def onion_peel(lv, prm, level_index):
    """Algorithm 3 at the coarsest level: onion_layer until H' is empty,
    starting from H' = H. A layer voxel that no patch centred outside H'
    covers is kept in H' for the next layer."""
    Hp = lv.hole.copy()
    n_layer = 0
    evals = 0
    while Hp.any():
        new_Hp, ev = onion_layer(lv, prm, level_index, n_layer, Hp)
        evals += ev
        if new_Hp.sum() == Hp.sum():
            raise RuntimeError("onion peel made no progress")
        Hp = new_Hp
        n_layer += 1
    lv.stats["onion_layers"] = n_layer
    lv.stats["onion_evals"] = evals
    return n_layer


def _outer_count(prm, idx_from_coarsest):
    if prm.fixed_outer is None:
        return None
    if isinstance(prm.fixed_outer, int):
        return prm.fixed_outer
    return prm.fixed_outer[idx_from_coarsest]


def iterate_level(lv, prm, level_index, n_outer=None, start_call=0):
    """The inner loop of Algorithm 4 at one level: ANN search, then
    reconstruction of u and T, until e <= stop or max_outer iterations
    (or exactly n_outer iterations when given). Iteration k uses call index
    start_call + k, and the cap of Sec. 3.7 counts the level's iterations
    from call 0, so a loop resumed at start_call stops where the whole loop
    would."""
    nH = int(lv.hole.sum())
    k = 0
    e = math.inf
    evals = 0
    es = []
    while True:
        if n_outer is not None:
            if k >= n_outer:
                break
        elif not (e > prm.stop and start_call + k < prm.max_outer):
            break
        evals += ann(lv.x, lv.htilde, lv.dtilde, lv.phi, lv.d2, n_pm=prm.n_pm,
                     schedule=prm.schedule, rho=prm.rho, key=prm.key,
                     tag_base=tag(PURPOSE_SEARCH, level_index, start_call + k), clip=prm.clip,
                     rs_mode=prm.rs_mode, sub_sweeps=prm.sub_sweeps)
        lv.x, change = vote(lv.x, lv.hole, lv.htilde, lv.phi, lv.d2, weighted=prm.weighted,
                            n_diff=3)
        e = change / (3.0 * max(nH, 1))
        es.append(e)
        k += 1
    lv.stats.setdefault("outer", []).append(k)
    lv.stats.setdefault("e", []).extend(es)
    lv.stats["evals"] = lv.stats.get("evals", 0) + evals
    return k


def provisional_fill(coarse_x, fine_x, fine_hole, tsub=False):
    """The first half of the level transition (Sec. 3.6): every occluded voxel
    (x, y, t) of the finer level takes, in place, the value of its coarse
    parent (x // 2, y // 2, t), or (x // 2, y // 2, t // 2) with temporal
    subsampling, so that the distances of Eq. 5 have a video to compare."""
    tt, yy, xx = np.nonzero(fine_hole)
    fine_x[tt, yy, xx] = coarse_x[tt // 2 if tsub else tt, yy // 2, xx // 2]
    return fine_x


def next_level(coarse, fine, prm, fine_index):
    """Level transition of Algorithm 4: phi^{l-1} = UpSample(phi^l, 2); the
    finer occluded voxels first take their coarse parent's value (the
    distances of Eq. 5 need a video to compare); distances; reconstruction of
    u and T at the finer level (Eq. 4/5, Eq. 9)."""
    fine.phi = upsample_nnf(coarse.phi, fine.htilde, fine.dtilde, prm.key,
                            tag(PURPOSE_UPSAMPLE, fine_index), prm.clip, prm.time_subsample)
    fine.d2 = np.full(fine.hole.shape, np.inf, prm.d2_dtype)
    provisional_fill(coarse.x, fine.x, fine.hole, prm.time_subsample)
    ev = _rescore(fine, prm)
    fine.x, _ = vote(fine.x, fine.hole, fine.htilde, fine.phi, fine.d2,
                     weighted=prm.weighted, n_diff=3)
    fine.stats["transition_evals"] = ev


def inpaint(rgb, mask, levels, use_texture=True, prm=None, return_levels=False):
    """Algorithm 4 (the affine realignment of Algorithm 2 is not part of this
    path). Returns the inpainted RGB video float32 [T][H][W][3]."""
    prm = prm or Params()
    pyr = build_pyramid(rgb, mask, levels, use_texture, prm.lam, prm.time_subsample)
    L = levels
    top = pyr[L - 1]
    if top.dtilde.sum() == 0:
        raise ValueError("no valid source patch at the coarsest level")
    top.phi = init_nnf(top.htilde, top.dtilde, prm.key, tag(PURPOSE_INIT, L - 1), prm.clip)
    top.d2 = np.full(top.hole.shape, np.inf, prm.d2_dtype)
    onion_peel(top, prm, L - 1)
    before_final = None
    for i, lv_index in enumerate(range(L - 1, -1, -1)):
        lv = pyr[lv_index]
        iterate_level(lv, prm, lv_index, n_outer=_outer_count(prm, i))
        if lv_index == 0:
            before_final = lv.x.copy()
            out = final(lv.x, lv.hole, lv.phi, lv.d2)
        else:
            next_level(lv, pyr[lv_index - 1], prm, lv_index - 1)
    rgb_out = np.ascontiguousarray(out[..., :3])
    # known voxels are returned as given
    keep = ~mask.astype(bool)
    rgb_out[keep] = _c(rgb, np.float32)[keep]
    if return_levels:
        return rgb_out, pyr, before_final
    return rgb_out
