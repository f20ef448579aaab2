"""Thin ctypes binding of the C ABI declared in ``include/vi.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libvi.so``. Loading fails loudly when the library has not been
built; there is no fallback implementation.

Arrays: numpy arrays are host memory (``ptr_is_device = 0``); torch CUDA
tensors are passed by ``data_ptr()`` as device memory (``ptr_is_device = 1``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

VI_OK = 0
STATUS = {0: "VI_OK", 1: "VI_ERR_ARG", 2: "VI_ERR_OOM", 3: "VI_ERR_CUDA", 4: "VI_ERR_TIMEOUT",
          5: "VI_ERR_NO_SOURCE", 6: "VI_ERR_STATE", 7: "VI_ERR_NO_DEVICE", 8: "VI_ERR_TOO_LARGE"}

# every entry point declared in include/vi.h
EXPORTS = [
    "vi_config_default", "vi_ctx_create", "vi_ctx_destroy", "vi_last_error", "vi_auto_levels",
    "vi_footprint_bytes", "vi_upload", "vi_build_pyramid", "vi_init_nnf", "vi_onion_peel",
    "vi_onion_layer", "vi_patch_dist_partial", "vi_prepare", "vi_rescore", "vi_ann", "vi_reconstruct", "vi_iterate", "vi_next_level",
    "vi_final", "vi_run", "vi_energy", "vi_level_info", "vi_get_channels", "vi_set_channels",
    "vi_get_nnf", "vi_set_nnf", "vi_get_masks", "vi_patch_dist", "vi_fetch_result",
    "vi_profile", "vi_get_stats", "vi_energy_noalloc", "vi_tune_export", "vi_tune_import",
    "vi_realign_last_error", "vi_affine_levels", "vi_affine_estimate", "vi_affine_to_reference",
    "vi_affine_align", "vi_affine_unwarp",
    "vi_server_create", "vi_server_submit", "vi_server_poll", "vi_server_wait", "vi_server_release",
    "vi_server_info", "vi_server_destroy", "vi_run_slabs", "vi_slabs_last_error",
    "vi_state_bytes", "vi_save_state", "vi_load_state", "vi_resume", "vi_iteration_log",
    "vi_batch_create", "vi_batch_destroy", "vi_batch_last_error", "vi_batch_add", "vi_batch_step",
    "vi_batch_run", "vi_batch_poll", "vi_batch_fetch", "vi_batch_remove", "vi_batch_clip_stats",
    "vi_batch_get_stats", "vi_batch_screen_stats", "vi_batch_profile", "vi_batch_step_time",
    "vi_batch_clip_ctx", "vi_batch_add_many",
]


class ViConfig(C.Structure):
    _fields_ = [("lambda_", C.c_float), ("n_pm", C.c_int), ("rho", C.c_float),
                ("levels", C.c_int), ("max_outer", C.c_int), ("stop", C.c_float),
                ("weighted", C.c_int), ("use_texture", C.c_int), ("storage", C.c_int),
                ("seed", C.c_uint64), ("clip", C.c_uint32), ("lanes_per_target", C.c_int),
                ("stream_priority", C.c_int), ("rs_mode", C.c_int), ("sub_sweeps", C.c_int),
                ("time_subsample", C.c_int), ("mem_limit", C.c_size_t)]


class ViStats(C.Structure):
    _fields_ = [("evals", C.c_ulonglong), ("step_evals", C.c_ulonglong),
                ("step_gathered", C.c_ulonglong), ("step_gathered_h", C.c_ulonglong),
                ("screened", C.c_ulonglong), ("screen_passed", C.c_ulonglong),
                ("step_launches", C.c_ulonglong), ("step_ms", C.c_double),
                ("step_timed", C.c_ulonglong), ("outer", C.c_int * 16),
                ("onion_layers", C.c_int), ("levels", C.c_int), ("launches", C.c_ulonglong)]


class ViError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load libvi.so (building it first only when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        _build.build()
    lib = C.CDLL(path)
    _declare(lib)
    _lib = lib
    return lib


def _declare(L):
    vp, i, f, d, ll = C.c_void_p, C.c_int, C.c_float, C.c_double, C.c_longlong
    P = C.POINTER
    L.vi_config_default.argtypes = [P(ViConfig)]
    L.vi_config_default.restype = None
    L.vi_ctx_create.argtypes = [P(ViConfig), vp, P(vp)]
    L.vi_ctx_destroy.argtypes = [vp]
    L.vi_ctx_destroy.restype = None
    L.vi_last_error.argtypes = [vp]
    L.vi_last_error.restype = C.c_char_p
    L.vi_auto_levels.argtypes = [vp, i, i, i]
    L.vi_footprint_bytes.argtypes = [P(ViConfig), i, i, i, ll]
    L.vi_footprint_bytes.restype = C.c_size_t
    L.vi_upload.argtypes = [vp, vp, vp, i, i, i, i]
    for name in ("vi_build_pyramid", "vi_onion_peel", "vi_prepare", "vi_final", "vi_run"):
        getattr(L, name).argtypes = [vp]
    L.vi_init_nnf.argtypes = [vp, i]
    L.vi_rescore.argtypes = [vp, i]
    L.vi_ann.argtypes = [vp, i, i]
    L.vi_reconstruct.argtypes = [vp, i, P(f)]
    L.vi_iterate.argtypes = [vp, i, i, i, P(i), P(f)]
    L.vi_next_level.argtypes = [vp, i]
    L.vi_energy.argtypes = [vp, i, P(d), P(d)]
    L.vi_level_info.argtypes = [vp, i, P(i), P(i), P(i), P(i), P(ll), P(ll), P(ll)]
    L.vi_get_channels.argtypes = [vp, i, vp, i]
    L.vi_set_channels.argtypes = [vp, i, vp, i]
    L.vi_get_nnf.argtypes = [vp, i, vp, vp]
    L.vi_set_nnf.argtypes = [vp, i, vp, vp]
    L.vi_get_masks.argtypes = [vp, i, vp]
    L.vi_patch_dist.argtypes = [vp, i, vp, i, vp]
    L.vi_patch_dist_partial.argtypes = [vp, i, vp, i, vp, vp]
    L.vi_onion_layer.argtypes = [vp, i, vp, vp, P(i)]
    L.vi_fetch_result.argtypes = [vp, vp, i]
    L.vi_profile.argtypes = [vp, i]
    L.vi_get_stats.argtypes = [vp, P(ViStats)]
    L.vi_energy_noalloc.argtypes = [vp, i, vp, vp, i, i, i, vp, vp]
    L.vi_tune_export.argtypes = [C.c_char_p, i]
    L.vi_tune_export.restype = i
    L.vi_tune_import.argtypes = [C.c_char_p]
    L.vi_server_create.argtypes = [C.c_size_t, i, P(vp)]
    L.vi_server_submit.argtypes = [vp, P(ViConfig), vp, vp, i, i, i, i, vp, P(C.c_uint64)]
    L.vi_server_poll.argtypes = [vp, C.c_uint64, P(i)]
    L.vi_server_wait.argtypes = [vp, C.c_uint64, d, P(i)]
    L.vi_server_release.argtypes = [vp, C.c_uint64, C.c_char_p, i]
    L.vi_server_info.argtypes = [vp, P(i), P(i), P(C.c_size_t)]
    L.vi_server_destroy.argtypes = [vp]
    L.vi_server_destroy.restype = None
    L.vi_realign_last_error.argtypes = []
    L.vi_realign_last_error.restype = C.c_char_p
    L.vi_affine_levels.argtypes = [i, i]
    L.vi_affine_estimate.argtypes = [vp, vp, i, i, i, i, i, i, vp, vp]
    L.vi_affine_to_reference.argtypes = [vp, i, vp]
    L.vi_affine_align.argtypes = [vp, vp, i, i, i, vp, vp, vp, i, vp]
    L.vi_affine_unwarp.argtypes = [vp, vp, vp, i, i, i, vp, vp, i, vp]
    L.vi_iteration_log.argtypes = [vp, i, P(i), P(i), P(C.c_float), P(C.c_ulonglong)]
    L.vi_iteration_log.restype = i
    L.vi_state_bytes.argtypes = [vp, i]
    L.vi_state_bytes.restype = C.c_size_t
    L.vi_save_state.argtypes = [vp, i, vp, C.c_size_t]
    L.vi_load_state.argtypes = [vp, i, vp, C.c_size_t]
    L.vi_resume.argtypes = [vp, i, i]
    L.vi_run_slabs.argtypes = [P(ViConfig), vp, vp, i, i, i, i, i, vp, P(ViStats), P(C.c_ulonglong), vp, P(i)]
    L.vi_slabs_last_error.argtypes = []
    L.vi_slabs_last_error.restype = C.c_char_p
    ull = C.c_ulonglong
    L.vi_batch_create.argtypes = [P(ViConfig), vp, P(vp)]
    L.vi_batch_destroy.argtypes = [vp]
    L.vi_batch_destroy.restype = None
    L.vi_batch_last_error.argtypes = [vp]
    L.vi_batch_last_error.restype = C.c_char_p
    L.vi_batch_add.argtypes = [vp, P(ViConfig), vp, vp, i, i, i, i, P(i)]
    L.vi_batch_step.argtypes = [vp, P(i)]
    L.vi_batch_run.argtypes = [vp]
    L.vi_batch_poll.argtypes = [vp, i, P(i), P(i)]
    L.vi_batch_fetch.argtypes = [vp, i, vp, i]
    L.vi_batch_remove.argtypes = [vp, i]
    L.vi_batch_clip_stats.argtypes = [vp, i, P(ViStats)]
    L.vi_batch_clip_ctx.argtypes = [vp, i, P(vp), P(i)]
    L.vi_batch_add_many.argtypes = [vp, i, vp, vp, vp, P(i), P(i), P(i), i, i, P(i), P(i)]
    L.vi_batch_get_stats.argtypes = [vp, P(ull), P(ull), P(ull)]
    L.vi_batch_screen_stats.argtypes = [vp, P(ull), P(ull), P(ull)]
    L.vi_batch_profile.argtypes = [vp, i]
    L.vi_batch_step_time.argtypes = [vp, P(d), P(ull)]


def default_config(**kw):
    cfg = ViConfig()
    load().vi_config_default(C.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, "lambda_" if k == "lam" else k, v)
    return cfg


def _ptr(a):
    """(address, is_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous, "array must be C-contiguous"
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


class Context:
    """One inpainting context (``vi_ctx``); methods mirror the C entry points."""

    def __init__(self, cfg=None, stream=None, **kw):
        self.lib = load()
        if cfg is None:
            cfg = default_config(**kw)
        h = C.c_void_p()
        st = self.lib.vi_ctx_create(C.byref(cfg), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != VI_OK:
            raise ViError(st, "vi_ctx_create failed")
        self.h = h
        self.cfg = cfg

    def close(self):
        if getattr(self, "h", None):
            if not getattr(self, "borrowed", False):
                self.lib.vi_ctx_destroy(self.h)
            self.h = None

    @classmethod
    def borrow(cls, lib, h):
        """A view of a context the library owns (a batch clip's): the same
        methods, and close() leaves the context alone."""
        obj = cls.__new__(cls)
        obj.lib, obj.h, obj.cfg, obj.borrowed = lib, h, None, True
        return obj

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        if st != VI_OK:
            raise ViError(st, self.lib.vi_last_error(self.h).decode(errors="replace"))

    # -- whole method and steps -------------------------------------------
    def upload(self, rgb, mask):
        if isinstance(rgb, np.ndarray):
            rgb = np.ascontiguousarray(rgb, dtype=np.float32)
        if isinstance(mask, np.ndarray):
            mask = np.ascontiguousarray(mask, dtype=np.uint8)
        self._keep = (rgb, mask)
        pr, dr = _ptr(rgb)
        pm, dm = _ptr(mask)
        assert dr == dm, "rgb and mask must both be host or both be device memory"
        T, H, W = mask.shape[:3]
        self._ck(self.lib.vi_upload(self.h, pr, pm, W, H, T, dr))

    def build_pyramid(self):
        self._ck(self.lib.vi_build_pyramid(self.h))

    def init_nnf(self, level):
        self._ck(self.lib.vi_init_nnf(self.h, level))

    def onion_peel(self):
        self._ck(self.lib.vi_onion_peel(self.h))

    def onion_layer(self, layer, hprime=None):
        """One layer of Algorithm 3 (vi_onion_layer). hprime: uint8 [T][H][W]
        of the coarsest level (None: continue from the context's own H').
        Returns (H' after the layer, its size)."""
        info = self.level_info(self.stats()["levels"] - 1)
        out = np.zeros((info["T"], info["H"], info["W"]), np.uint8)
        hin = None
        if hprime is not None:
            hin = np.ascontiguousarray(hprime, np.uint8)
            assert hin.shape == out.shape
        left = C.c_int(0)
        self._ck(self.lib.vi_onion_layer(self.h, int(layer), hin.ctypes.data if hin is not None else None,
                                         out.ctypes.data, C.byref(left)))
        return out, left.value

    def prepare(self):
        self._ck(self.lib.vi_prepare(self.h))

    def rescore(self, level):
        self._ck(self.lib.vi_rescore(self.h, level))

    def ann(self, level, call=0):
        self._ck(self.lib.vi_ann(self.h, level, call))

    def reconstruct(self, level, want_e=True):
        e = C.c_float(0.0)
        self._ck(self.lib.vi_reconstruct(self.h, level, C.byref(e) if want_e else None))
        return e.value if want_e else None

    def iterate(self, level, n_outer=-1, first_call=0):
        n = C.c_int(0)
        e = C.c_float(0.0)
        self._ck(self.lib.vi_iterate(self.h, level, n_outer, first_call, C.byref(n), C.byref(e)))
        return n.value, e.value

    def next_level(self, level):
        self._ck(self.lib.vi_next_level(self.h, level))

    def final(self):
        self._ck(self.lib.vi_final(self.h))

    def run(self):
        self._ck(self.lib.vi_run(self.h))

    def energy(self, level):
        a, b = C.c_double(0.0), C.c_double(0.0)
        self._ck(self.lib.vi_energy(self.h, level, C.byref(a), C.byref(b)))
        return a.value, b.value

    # -- state access ---------------------------------------------------------
    def level_info(self, level):
        W, H, T, Cn = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        nh, nt, ns = C.c_longlong(), C.c_longlong(), C.c_longlong()
        self._ck(self.lib.vi_level_info(self.h, level, C.byref(W), C.byref(H), C.byref(T),
                                        C.byref(Cn), C.byref(nh), C.byref(nt), C.byref(ns)))
        return dict(W=W.value, H=H.value, T=T.value, C=Cn.value, n_hole=nh.value,
                    n_target=nt.value, n_source=ns.value)

    def get_channels(self, level, out=None):
        info = self.level_info(level)
        if out is None:
            out = np.empty((info["T"], info["H"], info["W"], info["C"]), np.float32)
        p, dev = _ptr(out)
        self._ck(self.lib.vi_get_channels(self.h, level, p, dev))
        return out

    def set_channels(self, level, x):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float32)
        p, dev = _ptr(x)
        self._ck(self.lib.vi_set_channels(self.h, level, p, dev))

    def get_nnf(self, level):
        info = self.level_info(level)
        phi = np.zeros((info["T"], info["H"], info["W"], 3), np.int32)
        d2 = np.zeros((info["T"], info["H"], info["W"]), np.float32)
        self._ck(self.lib.vi_get_nnf(self.h, level, phi.ctypes.data, d2.ctypes.data))
        return phi, d2

    def set_nnf(self, level, phi=None, d2=None):
        pp = np.ascontiguousarray(phi, np.int32) if phi is not None else None
        dd = np.ascontiguousarray(d2, np.float32) if d2 is not None else None
        self._ck(self.lib.vi_set_nnf(self.h, level, pp.ctypes.data if pp is not None else None,
                                     dd.ctypes.data if dd is not None else None))

    def get_masks(self, level):
        info = self.level_info(level)
        code = np.zeros((info["T"], info["H"], info["W"]), np.uint8)
        self._ck(self.lib.vi_get_masks(self.h, level, code.ctypes.data))
        return code

    def patch_dist_partial(self, level, pairs, excl):
        """Eq. 11 distances for (px, py, pt, sx, sy, st) pairs, target voxels
        with excl != 0 left out (vi_patch_dist_partial)."""
        pairs = np.ascontiguousarray(pairs, np.int32).reshape(-1, 6)
        ex = np.ascontiguousarray(excl, np.uint8)
        out = np.zeros(len(pairs), np.float32)
        self._ck(self.lib.vi_patch_dist_partial(self.h, level, pairs.ctypes.data, len(pairs), ex.ctypes.data,
                                                out.ctypes.data))
        return out

    def patch_dist(self, level, pairs):
        pairs = np.ascontiguousarray(pairs, np.int32).reshape(-1, 6)
        out = np.zeros(len(pairs), np.float32)
        self._ck(self.lib.vi_patch_dist(self.h, level, pairs.ctypes.data, len(pairs),
                                        out.ctypes.data))
        return out

    def fetch_result(self, out=None):
        if out is None:
            info = self.level_info(0)
            out = np.empty((info["T"], info["H"], info["W"], 3), np.float32)
        p, dev = _ptr(out)
        self._ck(self.lib.vi_fetch_result(self.h, p, dev))
        return out

    def iteration_log(self):
        """Per iteration that computed e: level, call, e and the evaluation
        count after it (vi_iteration_log)."""
        n = self.lib.vi_iteration_log(self.h, 0, None, None, None, None)
        lv, ca = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))()
        e, ev = (C.c_float * max(n, 1))(), (C.c_ulonglong * max(n, 1))()
        self.lib.vi_iteration_log(self.h, n, lv, ca, e, ev)
        return [dict(level=lv[i], call=ca[i], e=e[i], evals=ev[i]) for i in range(n)]

    def save_state(self, level):
        """The level's state between two iterations (vi_save_state), as bytes."""
        n = self.lib.vi_state_bytes(self.h, level)
        if n == 0:
            raise ViError(1, "vi_state_bytes: bad level or no pyramid")
        buf = C.create_string_buffer(n)
        self._ck(self.lib.vi_save_state(self.h, level, buf, n))
        return buf.raw

    def load_state(self, level, state):
        buf = C.create_string_buffer(bytes(state), len(state))
        self._ck(self.lib.vi_load_state(self.h, level, buf, len(state)))

    def resume(self, level, first_call):
        """The rest of Algorithm 4 from call first_call of level (vi_resume)."""
        self._ck(self.lib.vi_resume(self.h, level, first_call))

    def profile(self, enable=True):
        self._ck(self.lib.vi_profile(self.h, 1 if enable else 0))

    def stats(self):
        s = ViStats()
        self._ck(self.lib.vi_get_stats(self.h, C.byref(s)))
        return _stats_dict(s)


def _stats_dict(s):
    return dict(evals=s.evals, step_evals=s.step_evals, step_gathered=s.step_gathered,
                step_gathered_h=s.step_gathered_h, screened=s.screened, screen_passed=s.screen_passed,
                step_launches=s.step_launches, step_ms=s.step_ms, step_timed=s.step_timed,
                outer=list(s.outer), onion_layers=s.onion_layers, levels=s.levels,
                launches=s.launches)


class Batch:
    """A batch of clips (``vi_batch``): one launch per step for all of them."""

    def __init__(self, cfg=None, stream=None, **kw):
        self.lib = load()
        if cfg is None:
            cfg = default_config(**kw)
        self.cfg = cfg
        self.defaults = dict(kw)
        h = C.c_void_p()
        st = self.lib.vi_batch_create(C.byref(cfg), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != VI_OK:
            raise ViError(st, "vi_batch_create failed")
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.vi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        if st != VI_OK:
            raise ViError(st, self.lib.vi_batch_last_error(self.h).decode(errors="replace"))

    def add(self, rgb, mask, **job):
        """Adds and prepares a clip; job overrides the batch's config fields
        (seed, clip, levels, ...). Returns the clip id."""
        cfg = default_config(**{**self.defaults, **job})
        if isinstance(rgb, np.ndarray):
            rgb = np.ascontiguousarray(rgb, dtype=np.float32)
        if isinstance(mask, np.ndarray):
            mask = np.ascontiguousarray(mask, dtype=np.uint8)
        pr, dr = _ptr(rgb)
        pm, dm = _ptr(mask)
        assert dr == dm
        T, H, W = mask.shape[:3]
        cid = C.c_int(-1)
        self._ck(self.lib.vi_batch_add(self.h, C.byref(cfg), pr, pm, W, H, T, dr, C.byref(cid)))
        self._keep[cid.value] = (rgb, mask, (T, H, W))
        return cid.value

    def add_many(self, items, n_threads=0):
        """Adds clips at once (vi_batch_add_many: uploads and preparations
        run concurrently). items: (rgb, mask, job dict) per clip, all numpy
        or all CUDA tensors. Returns the ids; raises ViError when a clip
        fails (the others are added)."""
        n = len(items)
        if n == 0:
            return []
        cfgs = [default_config(**{**self.defaults, **job}) for _, _, job in items]
        cfg_ptrs = (C.c_void_p * n)(*[C.addressof(c) for c in cfgs])
        rgbs, masks, keep, dev = [], [], [], None
        Ws, Hs, Ts = (C.c_int * n)(), (C.c_int * n)(), (C.c_int * n)()
        for k, (rgb, mask, _) in enumerate(items):
            if isinstance(rgb, np.ndarray):
                rgb = np.ascontiguousarray(rgb, dtype=np.float32)
            if isinstance(mask, np.ndarray):
                mask = np.ascontiguousarray(mask, dtype=np.uint8)
            pr, dr = _ptr(rgb)
            pm, dm = _ptr(mask)
            assert dr == dm and (dev is None or dev == dr), "all host or all device buffers"
            dev = dr
            T, H, W = mask.shape[:3]
            Ws[k], Hs[k], Ts[k] = W, H, T
            rgbs.append(pr)
            masks.append(pm)
            keep.append((rgb, mask, (T, H, W)))
        ids = (C.c_int * n)()
        sts = (C.c_int * n)()
        st = self.lib.vi_batch_add_many(self.h, n, cfg_ptrs, (C.c_void_p * n)(*rgbs), (C.c_void_p * n)(*masks),
                                        Ws, Hs, Ts, int(dev), int(n_threads), ids, sts)
        for k in range(n):
            if ids[k] >= 0:
                self._keep[ids[k]] = keep[k]
        if st != VI_OK:
            err = ViError(st, self.lib.vi_batch_last_error(self.h).decode(errors="replace"))
            err.ids, err.statuses = list(ids), list(sts)   # the clips that were added
            raise err
        return list(ids)

    def step(self):
        n = C.c_int(0)
        self._ck(self.lib.vi_batch_step(self.h, C.byref(n)))
        return n.value

    def run(self):
        self._ck(self.lib.vi_batch_run(self.h))

    def poll(self, cid):
        done, level = C.c_int(0), C.c_int(0)
        self._ck(self.lib.vi_batch_poll(self.h, cid, C.byref(done), C.byref(level)))
        return done.value, level.value

    def fetch(self, cid, out=None):
        if out is None:
            T, H, W = self._keep[cid][2]
            out = np.empty((T, H, W, 3), np.float32)
        p, dev = _ptr(out)
        self._ck(self.lib.vi_batch_fetch(self.h, cid, p, dev))
        return out

    def remove(self, cid):
        self._ck(self.lib.vi_batch_remove(self.h, cid))
        self._keep.pop(cid, None)

    def clip_context(self, cid):
        """(context view, iteration index at its level) of a clip
        (vi_batch_clip_ctx), for injecting and reading its state."""
        h = C.c_void_p()
        call = C.c_int(0)
        self._ck(self.lib.vi_batch_clip_ctx(self.h, cid, C.byref(h), C.byref(call)))
        return Context.borrow(self.lib, h), call.value

    def clip_stats(self, cid):
        s = ViStats()
        self._ck(self.lib.vi_batch_clip_stats(self.h, cid, C.byref(s)))
        return _stats_dict(s)

    def stats(self):
        e, g, r = C.c_ulonglong(0), C.c_ulonglong(0), C.c_ulonglong(0)
        self._ck(self.lib.vi_batch_get_stats(self.h, C.byref(e), C.byref(g), C.byref(r)))
        ms, se = C.c_double(0.0), C.c_ulonglong(0)
        self._ck(self.lib.vi_batch_step_time(self.h, C.byref(ms), C.byref(se)))
        gh, sc, sp = C.c_ulonglong(0), C.c_ulonglong(0), C.c_ulonglong(0)
        self._ck(self.lib.vi_batch_screen_stats(self.h, C.byref(gh), C.byref(sc), C.byref(sp)))
        return dict(evals=e.value, gathered=g.value, rounds=r.value, step_ms=ms.value,
                    step_evals=se.value, gathered_h=gh.value, screened=sc.value, screen_passed=sp.value)

    def profile(self, enable=True):
        self._ck(self.lib.vi_batch_profile(self.h, 1 if enable else 0))


def tune_export():
    """The lanes-per-target autotuning table as text (see vi.h)."""
    L = load()
    n = L.vi_tune_export(None, 0)
    buf = C.create_string_buffer(n)
    L.vi_tune_export(buf, n)
    return buf.value.decode()


def tune_import(text):
    st = load().vi_tune_import(text.encode())
    if st != VI_OK:
        raise ViError(st, "vi_tune_import: malformed line")


class Server:
    """The native server (vi_server_*): submit() queues a request and returns
    its ticket; the arrays are kept alive here until the request is
    released."""

    def __init__(self, hbm_budget, max_slots=8, **defaults):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.vi_server_create(int(hbm_budget), int(max_slots), C.byref(h))
        if st != VI_OK:
            raise ViError(st, "vi_server_create failed")
        self.h = h
        self.defaults = dict(defaults)
        self._keep = {}

    def submit(self, rgb, mask, out=None, **job):
        if isinstance(rgb, np.ndarray):
            rgb = np.ascontiguousarray(rgb, np.float32)
        if isinstance(mask, np.ndarray):
            mask = np.ascontiguousarray(mask, np.uint8)
        T, H, W = mask.shape[:3]
        if out is None:
            out = np.empty((T, H, W, 3), np.float32)
        cfg = default_config(**{**self.defaults, **job})
        pr, dev = _ptr(rgb)
        pm, _ = _ptr(mask)
        po, _ = _ptr(out)
        t = C.c_uint64(0)
        st = self.lib.vi_server_submit(self.h, C.byref(cfg), pr, pm, W, H, T, dev, po, C.byref(t))
        if st != VI_OK:
            raise ViError(st, "vi_server_submit")
        self._keep[t.value] = (rgb, mask, out)
        return t.value

    def poll(self, ticket):
        d = C.c_int(0)
        st = self.lib.vi_server_poll(self.h, ticket, C.byref(d))
        if st != VI_OK:
            raise ViError(st, "vi_server_poll")
        return d.value

    def wait(self, ticket, timeout=-1.0):
        d = C.c_int(0)
        st = self.lib.vi_server_wait(self.h, ticket, float(timeout), C.byref(d))
        if st != VI_OK:
            raise ViError(st, "vi_server_wait")
        return d.value

    def release(self, ticket):
        """Returns the result array of a finished request and forgets it."""
        buf = C.create_string_buffer(512)
        st = self.lib.vi_server_release(self.h, ticket, buf, 512)
        keep = self._keep.pop(ticket, None)
        if st != VI_OK:
            raise ViError(st, "request failed: " + buf.value.decode(errors="replace"))
        return keep[2] if keep else None

    def info(self):
        q, r, b = C.c_int(0), C.c_int(0), C.c_size_t(0)
        self.lib.vi_server_info(self.h, C.byref(q), C.byref(r), C.byref(b))
        return dict(queued=q.value, running=r.value, bytes_in_use=b.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.vi_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rck(st, what):
    if st != VI_OK:
        raise ViError(st, f"{what}: " + load().vi_realign_last_error().decode(errors="replace"))


def affine_estimate(rgb, mask, levels=0, iters=10, stream=None):
    """Sec. 3.4: theta_{n,n+1} for every pair of successive frames, [T-1][6]."""
    rgb = np.ascontiguousarray(rgb, np.float32) if isinstance(rgb, np.ndarray) else rgb
    mask = np.ascontiguousarray(mask, np.uint8) if isinstance(mask, np.ndarray) else mask
    T, H, W = mask.shape[:3]
    out = np.zeros((max(T - 1, 0), 6), np.float64)
    pr, dr = _ptr(rgb)
    pm, dm = _ptr(mask)
    assert dr == dm
    _rck(load().vi_affine_estimate(pr, pm, W, H, T, dr, levels, iters, out.ctypes.data,
                                   C.c_void_p(stream) if stream else None), "vi_affine_estimate")
    return out


def affine_to_reference(theta_pairs, T):
    th = np.ascontiguousarray(theta_pairs, np.float64).reshape(-1, 6)
    out = np.zeros((T, 6), np.float64)
    _rck(load().vi_affine_to_reference(th.ctypes.data if th.size else None, T, out.ctypes.data),
         "vi_affine_to_reference")
    return out


def affine_align(rgb, mask, to_ref, rgb_out=None, mask_out=None, stream=None):
    """AlignVideo: (aligned rgb, aligned occlusion)."""
    rgb = np.ascontiguousarray(rgb, np.float32) if isinstance(rgb, np.ndarray) else rgb
    mask = np.ascontiguousarray(mask, np.uint8) if isinstance(mask, np.ndarray) else mask
    T, H, W = mask.shape[:3]
    tr = np.ascontiguousarray(to_ref, np.float64)
    pr, dev = _ptr(rgb)
    pm, _ = _ptr(mask)
    if rgb_out is None:
        rgb_out = np.empty((T, H, W, 3), np.float32)
        mask_out = np.empty((T, H, W), np.uint8)
    po, _ = _ptr(rgb_out)
    pq, _ = _ptr(mask_out)
    _rck(load().vi_affine_align(pr, pm, W, H, T, tr.ctypes.data, po, pq, dev,
                                C.c_void_p(stream) if stream else None), "vi_affine_align")
    return rgb_out, mask_out


def affine_unwarp(rgb, mask, aligned_result, to_ref, out=None, stream=None):
    """UnwarpVideo: the original video with its occluded pixels taken from
    the inpainted aligned video."""
    rgb = np.ascontiguousarray(rgb, np.float32) if isinstance(rgb, np.ndarray) else rgb
    mask = np.ascontiguousarray(mask, np.uint8) if isinstance(mask, np.ndarray) else mask
    res = np.ascontiguousarray(aligned_result, np.float32) if isinstance(aligned_result, np.ndarray) \
        else aligned_result
    T, H, W = mask.shape[:3]
    tr = np.ascontiguousarray(to_ref, np.float64)
    pr, dev = _ptr(rgb)
    pm, _ = _ptr(mask)
    pa, _ = _ptr(res)
    if out is None:
        out = np.empty((T, H, W, 3), np.float32)
    po, _ = _ptr(out)
    _rck(load().vi_affine_unwarp(pr, pm, pa, W, H, T, tr.ctypes.data, po, dev,
                                 C.c_void_p(stream) if stream else None), "vi_affine_unwarp")
    return out


def auto_levels(mask):
    mask = np.ascontiguousarray(mask, np.uint8)
    T, H, W = mask.shape
    return load().vi_auto_levels(mask.ctypes.data, W, H, T)


def run_slabs(rgb, mask, n_slabs, out=None, stream=None, devices=None, **cfg):
    """The whole inpainting with the finer levels split by frames over
    n_slabs contexts (vi_run_slabs): on one shared stream, or with devices
    (one device index per slab) on a stream of its own each. Returns (result,
    stats dict, bytes exchanged between the contexts)."""
    lib = load()
    if isinstance(rgb, np.ndarray):
        rgb = np.ascontiguousarray(rgb, np.float32)
    if isinstance(mask, np.ndarray):
        mask = np.ascontiguousarray(mask, np.uint8)
    T, H, W = mask.shape[:3]
    if out is None:
        out = np.empty((T, H, W, 3), np.float32)
    pr, dev = _ptr(rgb)
    pm, _ = _ptr(mask)
    po, _ = _ptr(out)
    cfgs = default_config(**cfg)
    st = ViStats()
    nbytes = C.c_ulonglong(0)
    devs = None
    if devices is not None:
        if len(devices) != int(n_slabs):
            raise ValueError("one device per slab")
        devs = (C.c_int * len(devices))(*[int(d) for d in devices])
    r = lib.vi_run_slabs(C.byref(cfgs), pr, pm, W, H, T, dev, int(n_slabs), po, C.byref(st), C.byref(nbytes),
                         C.c_void_p(stream) if stream else None, devs)
    if r != VI_OK:
        raise ViError(r, "vi_run_slabs: " + (lib.vi_slabs_last_error() or b"").decode(errors="replace"))
    return out, _stats_dict(st), nbytes.value


def inpaint(rgb, mask, realign=False, **cfg):
    """Run the whole method on one clip and return the inpainted video. With
    realign, Algorithm 4 as printed: AlignVideo (Sec. 3.4) first, inpainting
    in the aligned domain, UnwarpVideo last."""
    if not realign:
        with Context(**cfg) as ctx:
            ctx.upload(rgb, mask)
            ctx.run()
            return ctx.fetch_result()
    T = mask.shape[0]
    to_ref = affine_to_reference(affine_estimate(rgb, mask), T)
    al, al_mask = affine_align(rgb, mask, to_ref)
    with Context(**cfg) as ctx:
        ctx.upload(al, al_mask)
        ctx.run()
        res = ctx.fetch_result()
    return affine_unwarp(rgb, mask, res, to_ref)
