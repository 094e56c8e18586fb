"""FP64 CPU oracle (ctypes wrapper around ``csgs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it; the product path never imports it.  It shares no code
with the CUDA path.

Each function follows the paper's definitions (Sec. 3 "Scalar rendering function",
Eq. (sen), Algorithm 1); the C source states the details.  Functions that have no
independent pin are listed in the module docstring of the tests that pin the rest;
every function below is pinned (closed forms, invariants, published test vectors,
brute force on tiny cases) in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csgs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

RES_PIXEL, RES_SCENE, RES_CHANNEL, RES_TILE, RES_IMAGE = 0, 1, 2, 3, 4
VAR_L1, VAR_L2, VAR_NC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, IEEE FP64: no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_double), ("rho_max", ctypes.c_double), ("t_min", ctypes.c_double),
                ("cut2", ctypes.c_double), ("dilation", ctypes.c_double), ("clamp_fov", ctypes.c_double),
                ("obj_w", ctypes.c_double * 3), ("band_cut", ctypes.c_double), ("band_alpha", ctypes.c_double),
                ("band_tmin", ctypes.c_double), ("band_depth", ctypes.c_double),
                ("resolution", ctypes.c_int32), ("variant", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


def f32(x: float) -> float:
    """The value of x as the float32 number the library's options carry."""
    return float(np.float32(x))


@dataclasses.dataclass
class Opts:
    """Rendering/scoring conventions.  Defaults: the vanilla 3DGS rasteriser
    conventions the paper relies on (Sec. 3 and the 3-sigma footprint of the proof
    of Thm. 1).  The thresholds are the float32 numbers the library's option struct
    carries (e.g. 0.99f, 1e-4f), so both sides apply the same constants; this matters
    where the conventions meet exactly, e.g. (1 - 0.99)^2 = 1e-4.  The straddle bands
    mark queries whose decisions lie within a few times the FP32 error of the GPU
    path; they are test parameters, not part of the method."""
    alpha_min: float = f32(1.0 / 255.0)
    rho_max: float = f32(0.99)
    t_min: float = f32(1e-4)
    cut2: float = 9.0
    dilation: float = f32(0.3)
    clamp_fov: float = f32(1.3)
    obj_w: tuple = (1.0, 1.0, 1.0)
    band_cut: float = 5e-6     # relative band around the footprint cut
    band_alpha: float = 2e-6   # relative error of rho: band around alpha_min, feeds the T bound
    band_tmin: float = 4.0     # safety factor on the accumulated error bound of T near t_min
    band_depth: float = 2.5e-7  # relative depth difference treated as a tie
    resolution: int = RES_PIXEL
    variant: int = VAR_L1
    tile: int = 16

    def c(self) -> _Opts:
        o = _Opts()
        for f in dataclasses.fields(self):
            if f.name == "obj_w":
                o.obj_w = (ctypes.c_double * 3)(*self.obj_w)
            else:
                setattr(o, f.name, getattr(self, f.name))
        return o

    @staticmethod
    def pure(**kw) -> "Opts":
        """The paper's definitions with no rasteriser thresholds: alpha_min = 0,
        rho_max = 1, t_min = 0 (the footprint cut stays)."""
        d = dict(alpha_min=0.0, rho_max=1.0, t_min=0.0)
        d.update(kw)
        return Opts(**d)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.or_project.argtypes = [P, P, P, P, P]
        _lib.or_render.argtypes = [P, P, P, P, ctypes.c_int64, P, P, P, P, P, P]
        _lib.or_render_tiled.argtypes = [P, P, P, P, ctypes.c_int32, ctypes.c_int32, P, P, P]
        _lib.or_pixel_terms.argtypes = [P, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                        P, P, P, P, P]
        _lib.or_pixel_terms.restype = ctypes.c_int64
        _lib.or_score.argtypes = [P, P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P]
        _lib.or_sh_basis.argtypes = [ctypes.c_int, P, P]
        _lib.or_philox4x32_10.argtypes = [P, P, P]
        _lib.or_probabilities.argtypes = [P, ctypes.c_int64, P]
        _lib.or_probabilities.restype = ctypes.c_double
        _lib.or_cdf.argtypes = [P, ctypes.c_int64, P]
        _lib.or_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        _lib.or_uniform.restype = ctypes.c_uint64
        _lib.or_sample.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, P, P, P]
        _lib.or_sample.restype = ctypes.c_int64
        _lib.or_theorem2_m.argtypes = [ctypes.c_double] * 4
        _lib.or_theorem2_m.restype = ctypes.c_double
        _lib.or_transfer.argtypes = [P, P, P, P, P]
        _lib.or_score_pixels.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P]
        _lib.or_render_backward.argtypes = [P, P, P, P, P, P, P, P]
        _lib.or_mlp_nparam.restype = ctypes.c_int
        _lib.or_bf16.argtypes = [ctypes.c_double]
        _lib.or_bf16.restype = ctypes.c_double
        _lib.or_gelu.argtypes = [ctypes.c_double]
        _lib.or_gelu.restype = ctypes.c_double
        _lib.or_gelu_d.argtypes = [ctypes.c_double]
        _lib.or_gelu_d.restype = ctypes.c_double
        _lib.or_mlp_forward.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, P, P, P, P, P]
        _lib.or_mlp_backward.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int, P]
        _lib.or_mlp_backward.restype = ctypes.c_double
        _lib.or_adam.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int64]
        _lib.or_num_threads.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class SceneArrays:
    """Holds contiguous float32 copies of a scene and its C descriptor."""

    def __init__(self, scene):
        self.means = np.ascontiguousarray(scene.means, dtype=np.float32)
        self.log_scales = np.ascontiguousarray(scene.log_scales, dtype=np.float32)
        self.quats = np.ascontiguousarray(scene.quats, dtype=np.float32)
        self.opac = np.ascontiguousarray(scene.opacity_logits, dtype=np.float32)
        self.sh = np.ascontiguousarray(scene.sh, dtype=np.float32)
        self.n = self.means.shape[1]
        k = self.sh.shape[0]
        self.deg = {1: 0, 4: 1, 9: 2, 16: 3}[k]
        self.c = _Scene(self.n, self.deg, 0, self.means.ctypes.data, self.log_scales.ctypes.data,
                        self.quats.ctypes.data, self.opac.ctypes.data, self.sh.ctypes.data)


def _scene(scene):
    return scene if isinstance(scene, SceneArrays) else SceneArrays(scene)


def _cam(cam):
    return np.ascontiguousarray(cam, dtype=np.float32)


def num_threads() -> int:
    return lib().or_num_threads()


def project(scene, cam, opts: Opts | None = None, w=None) -> np.ndarray:
    """Per-Gaussian projection into one camera: [N, 16] = valid, mean x, mean y,
    conic (a, b, c), covariance (xx, xy, yy), depth, alpha, r, g, b, cam x, cam y."""
    sa = _scene(scene)
    opts = opts or Opts()
    out = np.zeros((sa.n, 16), dtype=np.float64)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    oc = opts.c()
    lib().or_project(ctypes.byref(sa.c), _ptr(_cam(cam)), ctypes.byref(oc), _ptr(w), _ptr(out))
    return out


def view_stats(scene, cams, opts: Opts | None = None) -> np.ndarray:
    """Per-Gaussian view statistics of the surrogate's inputs (not in the paper), from the
    projection above: [N, 3] = the number of views whose image the Gaussian's footprint
    reaches (valid projection, alpha >= alpha_min, and the bounding box
    |dx| <= sqrt(cut2 Sigma'_xx), |dy| <= sqrt(cut2 Sigma'_yy) of its ellipse overlapping
    the pixel centres' range [0, W - 1] x [0, H - 1]), the mean over those views of the
    ellipse's area pi cut2 sqrt(det Sigma'), and the maximum of that area."""
    opts = opts or Opts()
    cams = np.asarray(cams, dtype=np.float32).reshape(-1, 20)
    n = _scene(scene).n
    cnt, tot, mx = np.zeros(n), np.zeros(n), np.zeros(n)
    for cam in cams:
        P = project(scene, cam, opts)
        W, H = float(cam[16]), float(cam[17])
        rx, ry = np.sqrt(opts.cut2 * P[:, 6]), np.sqrt(opts.cut2 * P[:, 8])
        vis = ((P[:, 0] > 0) & (P[:, 10] >= opts.alpha_min) & (P[:, 1] + rx >= 0) & (P[:, 1] - rx <= W - 1)
               & (P[:, 2] + ry >= 0) & (P[:, 2] - ry <= H - 1))
        area = np.pi * opts.cut2 * np.sqrt(np.maximum(P[:, 6] * P[:, 8] - P[:, 7] ** 2, 0.0))
        cnt += vis
        tot += np.where(vis, area, 0.0)
        mx = np.maximum(mx, np.where(vis, area, 0.0))
    return np.stack([cnt, np.where(cnt > 0, tot / np.maximum(cnt, 1), 0.0), mx], 1)


def render(scene, cam, opts: Opts | None = None, w=None, pixels=None):
    """Render one camera (or the listed pixels).  Returns dict with rgb [H,W,3] (or
    [P,3]), T, n_terms, flags and the counters (violations, flagged pixels)."""
    sa = _scene(scene)
    opts = opts or Opts()
    cam = _cam(cam)
    W, H = int(cam[16]), int(cam[17])
    if pixels is not None:
        pixels = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        npix = pixels.shape[0]
        shape = (npix,)
    else:
        npix = W * H
        shape = (H, W)
    rgb = np.zeros(shape + (3,), dtype=np.float64)
    T = np.zeros(shape, dtype=np.float64)
    nt = np.zeros(shape, dtype=np.int32)
    fl = np.zeros(shape, dtype=np.uint8)
    cnt = np.zeros(2, dtype=np.int64)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    oc = opts.c()
    rc = lib().or_render(ctypes.byref(sa.c), _ptr(cam), ctypes.byref(oc), _ptr(w), npix, _ptr(pixels),
                         _ptr(rgb), _ptr(T), _ptr(nt), _ptr(fl), _ptr(cnt))
    if rc:
        raise MemoryError("oracle render failed")
    return dict(rgb=rgb, T=T, n_terms=nt, flags=fl, violations=int(cnt[0]), flagged=int(cnt[1]))


def render_tiled(scene, cam, tile_w: int, tile_h: int, opts: Opts | None = None, w=None):
    """The whole camera rendered by tiles of tile_w x tile_h pixels (each pixel composites
    only its tile's list).  Returns dict with rgb [H,W,3], T, n_terms."""
    sa = _scene(scene)
    opts = opts or Opts()
    cam = _cam(cam)
    W, H = int(cam[16]), int(cam[17])
    rgb = np.zeros((H, W, 3), dtype=np.float64)
    T = np.zeros((H, W), dtype=np.float64)
    nt = np.zeros((H, W), dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    oc = opts.c()
    rc = lib().or_render_tiled(ctypes.byref(sa.c), _ptr(cam), ctypes.byref(oc), _ptr(w), tile_w, tile_h, _ptr(rgb),
                               _ptr(T), _ptr(nt))
    if rc:
        raise MemoryError("oracle tiled render failed")
    return dict(rgb=rgb, T=T, n_terms=nt)


def pixel_terms(scene, cam, px: int, py: int, opts: Opts | None = None, w=None, cap: int = 1 << 16):
    """Ordered contributor list of one pixel: gid, rho, T, rgb per term, flag."""
    sa = _scene(scene)
    opts = opts or Opts()
    gid = np.zeros(cap, dtype=np.int64)
    rho = np.zeros(cap)
    T = np.zeros(cap)
    rgb = np.zeros((cap, 3))
    flag = np.zeros(1, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    oc = opts.c()
    n = lib().or_pixel_terms(ctypes.byref(sa.c), _ptr(_cam(cam)), ctypes.byref(oc), _ptr(w), px, py, cap,
                             _ptr(gid), _ptr(rho), _ptr(T), _ptr(rgb), _ptr(flag))
    n = min(int(n), cap)
    return dict(gid=gid[:n], rho=rho[:n], T=T[:n], rgb=rgb[:n], flag=int(flag[0]))


def score(scene, cams, opts: Opts | None = None, rows=None):
    """Sensitivity of every Gaussian (Eq. sen and the resolutions of Sec. 3).
    rows=(r0, r1) restricts every view to a band of rows (bounded samples)."""
    sa = _scene(scene)
    opts = opts or Opts()
    cams = np.ascontiguousarray(np.asarray(cams, dtype=np.float32).reshape(-1, 20))
    s = np.zeros(sa.n)
    sc = np.zeros(sa.n)
    touched = np.zeros(sa.n, dtype=np.uint8)
    cnt = np.zeros(5, dtype=np.int64)
    tot = np.zeros(2)
    r0, r1 = rows if rows is not None else (0, -1)
    oc = opts.c()
    rc = lib().or_score(ctypes.byref(sa.c), _ptr(cams), cams.shape[0], ctypes.byref(oc), r0, r1,
                        _ptr(s), _ptr(sc), _ptr(touched), _ptr(cnt), _ptr(tot))
    if rc:
        raise MemoryError("oracle score failed")
    return dict(s=s, s_clean=sc, touched=touched.astype(bool), queries=int(cnt[0]), flagged=int(cnt[1]),
                evaluated=int(cnt[2]), contributions=int(cnt[3]), pixels=int(cnt[4]), sumA=float(tot[0]),
                S=float(tot[1]))


def sh_basis(deg: int, d) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float64)
    out = np.zeros(16)
    lib().or_sh_basis(deg, _ptr(d), _ptr(out))
    return out[: (deg + 1) ** 2]


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def probabilities(s):
    s = np.ascontiguousarray(s, dtype=np.float64)
    p = np.zeros_like(s)
    S = lib().or_probabilities(_ptr(s), s.shape[0], _ptr(p))
    return p, S


def cdf(p) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    C = np.zeros(p.shape[0], dtype=np.uint64)
    lib().or_cdf(_ptr(p), p.shape[0], _ptr(C))
    return C


def uniform(seed: int, t: int, total: int) -> int:
    return int(lib().or_uniform(seed, t, total))


def sample(p, m: int, seed: int):
    """Algorithm 1 steps 4-5.  Returns dict(J [m], counts [N], w [N], idx (sorted
    distinct), w_sel, distinct)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    n = p.shape[0]
    J = np.zeros(max(m, 1), dtype=np.int32)
    counts = np.zeros(n, dtype=np.int32)
    w = np.zeros(n)
    d = lib().or_sample(_ptr(p), n, m, seed, _ptr(J), _ptr(counts), _ptr(w))
    idx = np.nonzero(counts)[0].astype(np.int32)
    return dict(J=J[:m], counts=counts, w=w, idx=idx, w_sel=w[idx], distinct=int(d))


def theorem2_m(S: float, eps: float, delta: float, n_queries: int) -> float:
    return lib().or_theorem2_m(S, eps, delta, float(n_queries))


def transfer(scene, cam, w, opts: Opts | None = None):
    """Per-pixel A, A_th (relaxed), A_w (true reduced render), gamma_q, min(1 - w rho)."""
    sa = _scene(scene)
    opts = opts or Opts.pure()
    cam = _cam(cam)
    W, H = int(cam[16]), int(cam[17])
    out = np.zeros((H, W, 11))
    w = np.ascontiguousarray(w, dtype=np.float64)
    oc = opts.c()
    lib().or_transfer(ctypes.byref(sa.c), _ptr(cam), ctypes.byref(oc), _ptr(w), _ptr(out))
    return dict(A=out[..., 0:3], A_th=out[..., 3:6], A_w=out[..., 6:9], gamma=out[..., 9], min_factor=out[..., 10])


def score_pixels(scene, cam, pixels, opts: Opts | None = None):
    """Per-pixel-resolution sensitivity over a list of (x, y) pixels of one camera."""
    sa = _scene(scene)
    opts = opts or Opts()
    pixels = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    s = np.zeros(sa.n)
    touched = np.zeros(sa.n, dtype=np.uint8)
    flags = np.zeros(pixels.shape[0], dtype=np.uint8)
    oc = opts.c()
    rc = lib().or_score_pixels(ctypes.byref(sa.c), _ptr(_cam(cam)), ctypes.byref(oc), pixels.shape[0], _ptr(pixels),
                               _ptr(s), _ptr(touched), _ptr(flags))
    if rc:
        raise MemoryError("oracle score_pixels failed")
    return dict(s=s, touched=touched.astype(bool), flags=flags.astype(bool))


# ---------------------------------------------------------------- surrogate MLP
MLP_IN, MLP_H = 64, 256


def mlp_nparam() -> int:
    return lib().or_mlp_nparam()


def mlp_split(P):
    """Views of a parameter block: W1 [256,64], b1, W2 [256,256], b2, w3, b3."""
    i = 0
    out = []
    for shape in ((MLP_H, MLP_IN), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_H,), (1,)):
        k = int(np.prod(shape))
        out.append(P[i:i + k].reshape(shape))
        i += k
    return out


def bf16(x: float) -> float:
    return lib().or_bf16(x)


def gelu(z: float) -> float:
    return lib().or_gelu(z)


def gelu_d(z: float) -> float:
    return lib().or_gelu_d(z)


def mlp_forward(P, X, emulate: bool = True):
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
    y = np.zeros(X.shape[0])
    lib().or_mlp_forward(_ptr(P), _ptr(X), X.shape[0], int(emulate), _ptr(y), None, None, None, None)
    return y


def mlp_backward(P, X, t, emulate: bool = True):
    """(loss, gradient block) of the mean squared error."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
    t = np.ascontiguousarray(t, dtype=np.float32)
    G = np.zeros_like(P)
    loss = lib().or_mlp_backward(_ptr(P), _ptr(X), _ptr(t), X.shape[0], int(emulate), _ptr(G))
    return loss, G


def adam(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    lib().or_adam(_ptr(p), _ptr(np.ascontiguousarray(g)), _ptr(m), _ptr(v), p.shape[0], lr, b1, b2, eps, step)


def render_backward(scene, cam, grad_rgb, opts: Opts | None = None, w=None):
    """Gradient of sum(grad_rgb * render) w.r.t. means [3,N], SH [(d+1)^2,3,N] and
    opacity logits [N] (scales and rotations fixed)."""
    sa = _scene(scene)
    opts = opts or Opts()
    gr = np.ascontiguousarray(grad_rgb, dtype=np.float64)
    gm = np.zeros((3, sa.n))
    gs = np.zeros(sa.sh.shape)
    gl = np.zeros(sa.n)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    oc = opts.c()
    rc = lib().or_render_backward(ctypes.byref(sa.c), _ptr(_cam(cam)), ctypes.byref(oc), _ptr(w), _ptr(gr), _ptr(gm),
                                  _ptr(gs), _ptr(gl))
    if rc:
        raise MemoryError("oracle render_backward failed")
    return gm, gs, gl
