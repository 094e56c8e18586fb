"""B300-native sensitivity scoring and coreset sampling for 3D Gaussian Splatting
pruning (arXiv 2607.02721, Sec. 3 and Algorithm 1).

This module is the thin Python binding of the C ABI in ``include/csgs.h``: it only
marshals arguments (tensor data pointers, the CUDA stream handle, ctypes structs)
into ``_lib/libcsgs.so``, where every step of the path runs in hand-written sm_103a
kernels.  PyTorch supplies device memory and streams.  There is no CPU fallback: if
the shared library is missing the import of the binding raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcsgs.so")

CSGS_OK = 0
CSGS_E_INVAL = -1
CSGS_E_NOMEM = -2
CSGS_E_CUDA = -3
CSGS_E_EMPTY = -4
CSGS_E_TIMEOUT = -5
CSGS_E_DEVICE_CHECK = -6
CSGS_NOALLOC_MAX_N = 262144
CSGS_MLP_PARAMS = 82689
RES_PIXEL = 0
RES_SCENE = 1
RES_CHANNEL = 2
RES_TILE = 3
RES_IMAGE = 4
VAR_L1 = 0
VAR_L2 = 1
VAR_NC = 2


class CsgsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"csgs error {status}: {msg}")
        self.status = status


class SceneDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("is_device", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("near_z", ctypes.c_float),
                ("pad", ctypes.c_float)]


class ScoreOpts(ctypes.Structure):
    _fields_ = [("resolution", ctypes.c_int32), ("variant", ctypes.c_int32), ("obj_w", ctypes.c_float * 3),
                ("alpha_min", ctypes.c_float), ("rho_max", ctypes.c_float), ("t_min", ctypes.c_float),
                ("cut2", ctypes.c_float), ("dilation", ctypes.c_float), ("clamp_fov", ctypes.c_float),
                ("view_batch", ctypes.c_int32), ("collect_stats", ctypes.c_int32), ("tile_shape", ctypes.c_int32),
                ("persist_ctas", ctypes.c_int32), ("accumulate", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("view_batch", ctypes.c_int32), ("sort_blocks", ctypes.c_int32), ("tile_shape", ctypes.c_int32),
                ("persist_ctas", ctypes.c_int32), ("probe_ms", ctypes.c_float)]


# Tile shapes (CSGS_TILE_*): 0 = the scene's autotuned shape (else 16x16).
TILE_AUTO, TILE_16X16, TILE_32X8, TILE_16X8, TILE_8X8 = 0, 1, 2, 3, 4
TILE_SHAPE_NAMES = {TILE_16X16: "16x16", TILE_32X8: "32x8", TILE_16X8: "16x8", TILE_8X8: "8x8"}


class Stats(ctypes.Structure):
    _fields_ = [("views", ctypes.c_int64), ("rays", ctypes.c_int64), ("instances", ctypes.c_int64),
                ("pairs_evaluated", ctypes.c_int64), ("pairs_hit", ctypes.c_int64),
                ("pairs_evaluated2", ctypes.c_int64), ("pairs_hit2", ctypes.c_int64), ("violations", ctypes.c_int64),
                ("capacity_retries", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("composite_launches", ctypes.c_int64), ("queries", ctypes.c_int64), ("score_ms", ctypes.c_double),
                ("project_ms", ctypes.c_double), ("sort_ms", ctypes.c_double), ("composite_ms", ctypes.c_double),
                ("entries_staged", ctypes.c_int64), ("entries_staged2", ctypes.c_int64),
                ("composite_busy_ms", ctypes.c_double), ("view_batches", ctypes.c_int64),
                ("warp_entries", ctypes.c_int64), ("warp_entries2", ctypes.c_int64),
                ("objective_sum", ctypes.c_double)]


EXPORTS = ("csgs_default_opts", "csgs_create", "csgs_destroy", "csgs_last_error", "csgs_load_scene",
           "csgs_load_scene_async",
           "csgs_free_scene", "csgs_set_queries", "csgs_score", "csgs_sample_coreset", "csgs_sample_coreset_p",
           "csgs_render", "csgs_sync", "csgs_get_stats", "csgs_debug_project", "csgs_kernel_launch_count",
           "csgs_sample_coreset_noalloc", "csgs_transfer", "csgs_theorem2_sample_size", "csgs_theorem3_eps",
           "csgs_debug_tc_gemm", "csgs_debug_tc_gemm_mn", "csgs_debug_tc_gemm_wait", "csgs_scale_scores", "csgs_total_sensitivity", "csgs_mlp_init", "csgs_mlp_set_params", "csgs_mlp_get_params", "csgs_mlp_forward",
           "csgs_mlp_gradient", "csgs_mlp_train", "csgs_view_stats", "csgs_features", "csgs_log_target",
           "csgs_surrogate_combine", "csgs_update_scene", "csgs_render_backward", "csgs_adam_update",
           "csgs_score_batch", "csgs_autotune", "csgs_debug_gelu", "csgs_log_ratio_mean", "csgs_log_residual_target",
           "csgs_surrogate_combine_prior")

_lib = None


def lib():
    """Load ``libcsgs.so`` (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is missing: run paper_2607_02721_b300.build.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    V, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    L.csgs_default_opts.argtypes = [V]
    L.csgs_default_opts.restype = None
    L.csgs_create.argtypes = [V, I32, V]
    L.csgs_destroy.argtypes = [V]
    L.csgs_destroy.restype = None
    L.csgs_last_error.argtypes = [V]
    L.csgs_last_error.restype = ctypes.c_char_p
    L.csgs_load_scene.argtypes = [V, V, V]
    L.csgs_load_scene_async.argtypes = [V, V, V]
    L.csgs_free_scene.argtypes = [V, I32]
    L.csgs_set_queries.argtypes = [V, I32, V, I32]
    L.csgs_score.argtypes = [V, I32, V, V, V]
    L.csgs_sample_coreset.argtypes = [V, V, I64, I64, U64, V, V, V]
    L.csgs_sample_coreset_p.argtypes = [V, V, I64, I64, U64, V, V, V, V]
    L.csgs_render.argtypes = [V, I32, I32, V, V, I64, V, V, V]
    L.csgs_sync.argtypes = [V]
    L.csgs_get_stats.argtypes = [V, V]
    L.csgs_debug_project.argtypes = [V, I32, I32, V, V]
    L.csgs_sample_coreset_noalloc.argtypes = [V, I64, I64, U64, V, V, V, V]
    L.csgs_transfer.argtypes = [V, I32, I32, V, V, I64, V, V]
    L.csgs_theorem2_sample_size.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, I64]
    L.csgs_theorem2_sample_size.restype = ctypes.c_double
    L.csgs_theorem3_eps.argtypes = [ctypes.c_double, ctypes.c_double]
    L.csgs_theorem3_eps.restype = ctypes.c_double
    L.csgs_debug_tc_gemm.argtypes = [V, V, V, V, I32, I32]
    L.csgs_debug_tc_gemm_mn.argtypes = [V, V, V, V, I32, I32]
    L.csgs_debug_tc_gemm_wait.argtypes = [V, V, V, V, I32, I32, ctypes.c_int64]
    L.csgs_scale_scores.argtypes = [V, V, ctypes.c_int64, ctypes.c_double]
    L.csgs_total_sensitivity.argtypes = [V, V, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    L.csgs_mlp_init.argtypes = [V, U64]
    L.csgs_mlp_set_params.argtypes = [V, V]
    L.csgs_mlp_get_params.argtypes = [V, V]
    L.csgs_mlp_forward.argtypes = [V, V, I64, V]
    L.csgs_mlp_gradient.argtypes = [V, V, V, I64, V, V]
    L.csgs_mlp_train.argtypes = [V, V, V, I64, I32, I32, ctypes.c_float, U64, V]
    L.csgs_view_stats.argtypes = [V, I32, V, V]
    L.csgs_features.argtypes = [V, I32, V, V, V]
    L.csgs_log_target.argtypes = [V, V, I64, ctypes.c_float, V]
    L.csgs_surrogate_combine.argtypes = [V, V, V, I64, ctypes.c_float, I32, V]
    L.csgs_log_ratio_mean.argtypes = [V, V, V, I64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.csgs_log_residual_target.argtypes = [V, V, V, I64, ctypes.c_float, ctypes.c_double, V]
    L.csgs_surrogate_combine_prior.argtypes = [V, V, V, V, I64, ctypes.c_float, ctypes.c_double, I32, V]
    L.csgs_update_scene.argtypes = [V, I32, V]
    L.csgs_render_backward.argtypes = [V, I32, I32, V, V, I64, V, V, V, V, V]
    L.csgs_adam_update.argtypes = [V, V, V, V, V, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   I32]
    L.csgs_score_batch.argtypes = [V, I32, V, V, V, V, I32]
    L.csgs_autotune.argtypes = [V, I32, V, I32, V]
    L.csgs_debug_gelu.argtypes = [V, V, I64, V]
    L.csgs_kernel_launch_count.argtypes = []
    L.csgs_kernel_launch_count.restype = I64
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is ctypes.c_int:  # default
            f.restype = ctypes.c_int32
    _lib = L
    return L


def default_opts(**kw) -> ScoreOpts:
    o = ScoreOpts()
    lib().csgs_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "obj_w":
            o.obj_w = (ctypes.c_float * 3)(*v)
        else:
            setattr(o, k, v)
    return o


def cameras(records) -> "ctypes.Array":
    """csgs_camera array from float records [V, 20] (see synth.CAMERA_FIELDS): the record's
    20 values are the struct's 20 four-byte fields in order, width and height as int32."""
    rec = np.asarray(records, dtype=np.float32).reshape(-1, 20)
    buf = np.ascontiguousarray(rec)
    buf = buf.copy()
    buf.view(np.int32)[:, 16:18] = rec[:, 16:18].astype(np.int32)
    buf[:, 19] = 0.0
    arr = (Camera * rec.shape[0])()
    ctypes.memmove(arr, buf.ctypes.data, buf.nbytes)
    return arr


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def theorem2_sample_size(S: float, eps_c: float, delta: float, n_queries: int) -> float:
    return float(lib().csgs_theorem2_sample_size(S, eps_c, delta, n_queries))


def theorem3_eps(gamma: float, eps_c: float) -> float:
    return float(lib().csgs_theorem3_eps(gamma, eps_c))


def kernel_launch_count() -> int:
    return int(lib().csgs_kernel_launch_count())


class Context:
    """One CUDA device + stream.  Methods mirror the csgs_* entry points.

    The library runs on ``self.stream`` (a torch stream, so tensors allocated for its
    outputs belong to it).  Before a call reads caller tensors the stream waits for the
    caller's current stream; after a call writes tensors the caller's stream waits for
    the library's stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        h = ctypes.c_void_p()
        r = lib().csgs_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if r != CSGS_OK:
            raise CsgsError(r, "csgs_create failed")
        self.h = h
        self._scenes = {}

    def _in(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _out(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _empty(self, shape, dtype):
        with self.torch.cuda.stream(self.stream):
            return self.torch.empty(shape, dtype=dtype, device=self.device)

    def _check(self, r):
        if r != CSGS_OK:
            raise CsgsError(r, lib().csgs_last_error(self.h).decode())
        return r

    def close(self):
        if getattr(self, "h", None):
            lib().csgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- scene and queries
    def load_scene(self, scene, on_device: bool = True) -> int:
        """Copy a scene (synth.Scene or an object with the same array attributes) into the
        context.  on_device: stage it through device tensors first (else the library
        copies from host memory)."""
        torch = self.torch
        arrs = [scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh]
        if on_device:
            with torch.cuda.stream(self.stream):
                keep = [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(self.device) for a in arrs]
            ptrs = [t.data_ptr() for t in keep]
        else:
            keep = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
            ptrs = [a.ctypes.data for a in keep]
        k = keep[4].shape[0]
        deg = {1: 0, 4: 1, 9: 2, 16: 3}[k]
        d = SceneDesc(int(keep[0].shape[1]), deg, 1 if on_device else 0, *ptrs)
        sid = ctypes.c_int32()
        self._in()
        self._check(lib().csgs_load_scene(self.h, ctypes.byref(d), ctypes.byref(sid)))
        self._scenes[sid.value] = int(keep[0].shape[1])
        return sid.value

    def load_scene_ptrs(self, n: int, sh_degree: int, ptrs, is_device: bool, asynchronous: bool = False) -> int:
        """Load a scene from raw attribute pointers.  asynchronous: csgs_load_scene_async
        (the sources must stay unchanged until the scene's first use)."""
        d = SceneDesc(n, sh_degree, 1 if is_device else 0, *ptrs)
        sid = ctypes.c_int32()
        self._in()
        fn = lib().csgs_load_scene_async if asynchronous else lib().csgs_load_scene
        self._check(fn(self.h, ctypes.byref(d), ctypes.byref(sid)))
        self._scenes[sid.value] = n
        return sid.value

    def scene_size(self, sid: int) -> int:
        """Number of Gaussians of a loaded scene."""
        return self._scenes[sid]

    def free_scene(self, sid: int):
        self._check(lib().csgs_free_scene(self.h, sid))
        self._scenes.pop(sid, None)

    def set_queries(self, sid: int, cams):
        arr = cams if isinstance(cams, ctypes.Array) else cameras(cams)
        self._check(lib().csgs_set_queries(self.h, sid, arr, len(arr)))

    # -- the hot path
    def score(self, sid: int, opts: ScoreOpts | None = None, out=None):
        """Sensitivities s (float32 [N] on the device) and S (host float)."""
        torch = self.torch
        n = self._scenes[sid]
        if out is None:
            out = self._empty(n, torch.float32)
        S = ctypes.c_double()
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_score(self.h, sid, ctypes.byref(opts), _ptr(out), ctypes.byref(S)))
        self._out()
        return out, S.value

    def scale_scores(self, s, factor: float):
        """s *= factor in place (library kernel, FP64 product rounded to FP32)."""
        self._in()
        self._check(lib().csgs_scale_scores(self.h, _ptr(s), s.numel(), float(factor)))
        self._out()
        return s

    def total_sensitivity(self, s) -> float:
        """S = sum of s in FP64 (the library's fixed-order reduction)."""
        S = ctypes.c_double()
        self._in()
        self._check(lib().csgs_total_sensitivity(self.h, _ptr(s), s.numel(), ctypes.byref(S)))
        self._out()
        return S.value

    def score_batch(self, sids, opts: ScoreOpts | None = None, outs=None, use_graph: bool = True):
        """Scores of several scenes in one submission (replayed as one CUDA graph after
        the first call).  Returns ([s_k], [S_k]).  Reuse `outs` to replay the graph."""
        torch = self.torch
        sids = [int(k) for k in sids]
        for k in sids:
            if k not in self._scenes:
                raise CsgsError(CSGS_E_INVAL, f"unknown scene id {k}")
        if outs is None:
            outs = [self._empty(self._scenes[k], torch.float32) for k in sids]
        ids = (ctypes.c_int32 * len(sids))(*sids)
        ptrs = (ctypes.c_void_p * len(sids))(*[o.data_ptr() for o in outs])
        S = (ctypes.c_double * len(sids))()
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_score_batch(self.h, len(sids), ids, ctypes.byref(opts), ptrs, S, int(use_graph)))
        self._out()
        return outs, list(S)

    def autotune(self, sid: int, opts: ScoreOpts | None = None, probe_views: int = 0) -> dict:
        """Tune a scene's view batch, sort grid, tile shape (a TILE_* value) and persistent
        compositing grid; returns the csgs_tuning fields as a dict."""
        out = Tuning()
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_autotune(self.h, sid, ctypes.byref(opts), probe_views, ctypes.byref(out)))
        self._out()
        return {f: getattr(out, f) for f, _ in Tuning._fields_}

    def sample_coreset(self, s, m: int, seed: int):
        torch = self.torch
        idx = self._empty(m, torch.int32)
        w = self._empty(m, torch.float32)
        nd = ctypes.c_int64()
        self._in()
        self._check(lib().csgs_sample_coreset(self.h, _ptr(s), s.numel(), m, seed, _ptr(idx), _ptr(w),
                                              ctypes.byref(nd)))
        self._out()
        return idx[: nd.value], w[: nd.value]

    def sample_coreset_p(self, p, m: int, seed: int, return_draws: bool = False):
        torch = self.torch
        idx = self._empty(m, torch.int32)
        w = self._empty(m, torch.float32)
        draws = self._empty(m, torch.int32) if return_draws else None
        nd = ctypes.c_int64()
        self._in()
        self._check(lib().csgs_sample_coreset_p(self.h, _ptr(p), p.numel(), m, seed, _ptr(idx), _ptr(w),
                                                ctypes.byref(nd), _ptr(draws)))
        self._out()
        if return_draws:
            return idx[: nd.value], w[: nd.value], draws
        return idx[: nd.value], w[: nd.value]

    def render(self, sid: int, view: int, idx=None, w=None, opts: ScoreOpts | None = None, H=None, W=None,
               with_T: bool = False, out=None):
        torch = self.torch
        if out is None:
            out = self._empty((H, W, 3), torch.float32)
        T = self._empty((H, W), torch.float32) if with_T else None
        n_sel = 0 if idx is None else idx.numel()
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_render(self.h, sid, view, _ptr(idx), _ptr(w), n_sel, ctypes.byref(opts), _ptr(out),
                                      _ptr(T)))
        self._out()
        return (out, T) if with_T else out

    def transfer(self, sid: int, view: int, idx, w, H: int, W: int, opts: ScoreOpts | None = None):
        """Per-pixel A, A_th, A_w, gamma_q, min(1 - w rho) of Sec. 3.3 ([H, W, 11])."""
        torch = self.torch
        out = self._empty((H, W, 11), torch.float32)
        opts = opts or default_opts(alpha_min=0.0, rho_max=1.0, t_min=0.0)
        self._in()
        self._check(lib().csgs_transfer(self.h, sid, view, _ptr(idx), _ptr(w), idx.numel(), ctypes.byref(opts),
                                        _ptr(out)))
        self._out()
        return out

    # -- surrogate model
    def debug_gelu(self, z):
        """[n, 2]: GELU and its derivative as the surrogate kernels evaluate them."""
        out = self._empty((z.numel(), 2), self.torch.float32)
        self._in()
        self._check(lib().csgs_debug_gelu(self.h, _ptr(z), z.numel(), _ptr(out)))
        self._out()
        return out

    def mlp_init(self, seed: int = 0):
        self._check(lib().csgs_mlp_init(self.h, seed))

    def mlp_set_params(self, P):
        self._in()
        self._check(lib().csgs_mlp_set_params(self.h, _ptr(P)))

    def mlp_get_params(self):
        P = self._empty(CSGS_MLP_PARAMS, self.torch.float32)
        self._check(lib().csgs_mlp_get_params(self.h, _ptr(P)))
        self._out()
        return P

    def mlp_forward(self, X):
        y = self._empty(X.shape[0], self.torch.float32)
        self._in()
        self._check(lib().csgs_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(y)))
        self._out()
        return y

    def mlp_gradient(self, X, t):
        G = self._empty(CSGS_MLP_PARAMS, self.torch.float32)
        loss = ctypes.c_float()
        self._in()
        self._check(lib().csgs_mlp_gradient(self.h, _ptr(X), _ptr(t), X.shape[0], _ptr(G), ctypes.byref(loss)))
        self._out()
        return G, loss.value

    def mlp_train(self, X, t, batch: int, steps: int, lr: float, seed: int = 0) -> float:
        loss = ctypes.c_float()
        self._in()
        self._check(lib().csgs_mlp_train(self.h, _ptr(X), _ptr(t), X.shape[0], batch, steps, lr, seed,
                                         ctypes.byref(loss)))
        self._out()
        return loss.value

    def view_stats(self, sid: int, opts: ScoreOpts | None = None):
        st = self._empty((self._scenes[sid], 3), self.torch.float32)
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_view_stats(self.h, sid, ctypes.byref(opts), _ptr(st)))
        self._out()
        return st

    def features(self, sid: int, stats, extra=None):
        X = self._empty((self._scenes[sid], 64), self.torch.bfloat16)
        self._in()
        self._check(lib().csgs_features(self.h, sid, _ptr(stats), _ptr(extra), _ptr(X)))
        self._out()
        return X

    def log_target(self, s, eps: float):
        t = self._empty(s.numel(), self.torch.float32)
        self._in()
        self._check(lib().csgs_log_target(self.h, _ptr(s), s.numel(), eps, _ptr(t)))
        self._out()
        return t

    def surrogate_combine(self, y, s_exact, eps: float, fill_only: bool = False):
        out = self._empty(y.numel(), self.torch.float32)
        self._in()
        self._check(lib().csgs_surrogate_combine(self.h, _ptr(y), _ptr(s_exact), y.numel(), eps, int(fill_only),
                                                 _ptr(out)))
        self._out()
        return out

    def log_ratio_mean(self, a, b):
        """(mean of log a - log b over the entries where both are > 0, their count)."""
        mean, cnt = ctypes.c_double(), ctypes.c_int64()
        self._in()
        self._check(lib().csgs_log_ratio_mean(self.h, _ptr(a), _ptr(b), a.numel(), ctypes.byref(mean),
                                              ctypes.byref(cnt)))
        return mean.value, cnt.value

    def log_residual_target(self, s, prior, eps: float, mu: float):
        t = self._empty(s.numel(), self.torch.float32)
        self._in()
        self._check(lib().csgs_log_residual_target(self.h, _ptr(s), _ptr(prior), s.numel(), eps, mu, _ptr(t)))
        self._out()
        return t

    def surrogate_combine_prior(self, y, prior, s_exact, eps: float, mu: float, fill_only: bool = False):
        out = self._empty(y.numel(), self.torch.float32)
        self._in()
        self._check(lib().csgs_surrogate_combine_prior(self.h, _ptr(y), _ptr(prior), _ptr(s_exact), y.numel(), eps,
                                                       mu, int(fill_only), _ptr(out)))
        self._out()
        return out

    # -- short recovery
    def update_scene(self, sid: int, means, log_scales, quats, opacity_logits, sh):
        """Overwrite a scene's attributes from device tensors (same shapes)."""
        k = sh.shape[0]
        deg = {1: 0, 4: 1, 9: 2, 16: 3}[k]
        d = SceneDesc(int(means.shape[1]), deg, 1, means.data_ptr(), log_scales.data_ptr(), quats.data_ptr(),
                      opacity_logits.data_ptr(), sh.data_ptr())
        self._in()
        self._check(lib().csgs_update_scene(self.h, sid, ctypes.byref(d)))

    def render_backward(self, sid: int, view: int, grad_rgb, g_means, g_sh, g_logit, idx=None, w=None, opts=None):
        n_sel = 0 if idx is None else idx.numel()
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_render_backward(self.h, sid, view, _ptr(idx), _ptr(w), n_sel, ctypes.byref(opts),
                                               _ptr(grad_rgb), _ptr(g_means), _ptr(g_sh), _ptr(g_logit)))
        self._out()

    def adam_update(self, p, g, m, v, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-15):
        self._in()
        self._check(lib().csgs_adam_update(self.h, _ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), lr, beta1, beta2,
                                           eps, step))
        self._out()

    def debug_tc_gemm(self, A, B):
        """C = A @ B^T on the tensor cores (A: [128, K] bf16, B: [N, K] bf16)."""
        torch = self.torch
        C = self._empty((A.shape[0], B.shape[0]), torch.float32)
        self._in()
        self._check(lib().csgs_debug_tc_gemm(self.h, _ptr(A), _ptr(B), _ptr(C), A.shape[1], B.shape[0]))
        self._out()
        return C

    def debug_tc_gemm_mn(self, At, Bt):
        """C = At^T @ Bt on the tensor cores with MN-major operands (At: [K, 128] bf16,
        Bt: [K, N] bf16)."""
        torch = self.torch
        C = self._empty((At.shape[1], Bt.shape[1]), torch.float32)
        self._in()
        self._check(lib().csgs_debug_tc_gemm_mn(self.h, _ptr(At), _ptr(Bt), _ptr(C), At.shape[0], Bt.shape[1]))
        self._out()
        return C

    def debug_tc_gemm_wait(self, A, B, first_wait_cycles: int):
        """debug_tc_gemm with the completion wait limited to ``first_wait_cycles`` clock
        cycles (0: one non-blocking test); raises CsgsError(CSGS_E_TIMEOUT) when it ran out."""
        torch = self.torch
        C = self._empty((A.shape[0], B.shape[0]), torch.float32)
        self._in()
        self._check(lib().csgs_debug_tc_gemm_wait(self.h, _ptr(A), _ptr(B), _ptr(C), A.shape[1], B.shape[0],
                                                  int(first_wait_cycles)))
        self._out()
        return C

    def debug_project(self, sid: int, view: int, opts: ScoreOpts | None = None):
        torch = self.torch
        n = self._scenes[sid]
        out = self._empty((n, 16), torch.float32)
        opts = opts or default_opts()
        self._in()
        self._check(lib().csgs_debug_project(self.h, sid, view, ctypes.byref(opts), _ptr(out)))
        self._out()
        return out

    def sync(self):
        self._check(lib().csgs_sync(self.h))

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().csgs_get_stats(self.h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}
