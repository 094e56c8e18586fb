"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only draws random scenes and cameras; it contains none of the
method's arithmetic (no projection, compositing, scoring or sampling).  Both the
GPU path and the CPU oracle receive the arrays it produces.

Scene layout (structure of arrays, float32):
  means        [3, N]   world-space centres mu_i
  log_scales   [3, N]   per-axis log standard deviations
  quats        [4, N]   rotation quaternions (w, x, y, z), unit length
  opacity_logits [N]    alpha_i = sigmoid(logit)
  sh           [(d+1)^2, 3, N]  real spherical-harmonic colour coefficients,
               coefficient-major then channel (R, G, B)

Camera layout (float32 record of 20 values, see ``CAMERA_FIELDS``): a pinhole
camera with row-major world-to-camera rotation R, translation t (p_cam = R p + t),
focal lengths fx, fy, principal point cx, cy, image width/height and near plane.
Camera axes follow the OpenCV convention: x right, y down, z forward.

The workloads mirror the paper's evaluation scenes (Sec. 4: pretrained 3DGS scenes
of a few million anisotropic Gaussians, SH degree 3, ~1-1.6 MP views), which are
not available here; the recipes below stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CAMERA_FIELDS = ("R0", "R1", "R2", "R3", "R4", "R5", "R6", "R7", "R8",
                 "t0", "t1", "t2", "fx", "fy", "cx", "cy", "W", "H", "near", "pad")


@dataclasses.dataclass
class Scene:
    means: np.ndarray          # float32 [3, N]
    log_scales: np.ndarray     # float32 [3, N]
    quats: np.ndarray          # float32 [4, N]
    opacity_logits: np.ndarray  # float32 [N]
    sh: np.ndarray             # float32 [(d+1)^2, 3, N]

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    @property
    def sh_degree(self) -> int:
        k = self.sh.shape[0]
        return {1: 0, 4: 1, 9: 2, 16: 3}[k]

    def subset(self, idx: np.ndarray) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.means[:, idx]),
                     np.ascontiguousarray(self.log_scales[:, idx]),
                     np.ascontiguousarray(self.quats[:, idx]),
                     np.ascontiguousarray(self.opacity_logits[idx]),
                     np.ascontiguousarray(self.sh[:, :, idx]))


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    return q.astype(np.float32)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Haar-random rotation from the QR factorisation of a Gaussian matrix."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def uniform_cube_scene(n: int, seed: int = 0) -> Scene:
    """Small exact-scoring workload: means uniform in [-1,1]^3, log-scales N(-4, 0.5^2)
    per axis, uniform random unit quaternions, opacity = sigmoid(N(0,1)), RGB uniform
    in [0,1] carried by the degree-0 SH coefficient.

    The DC coefficient is drawn uniform in [-sqrt(pi), sqrt(pi)], the range that the
    degree-0 basis value 1/(2 sqrt(pi)) plus the 0.5 colour offset maps onto [0, 1].
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (3, n)).astype(np.float32)
    log_scales = rng.normal(-4.0, 0.5, (3, n)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n).astype(np.float32)
    sqrt_pi = math.sqrt(math.pi)
    sh = rng.uniform(-sqrt_pi, sqrt_pi, (1, 3, n)).astype(np.float32)
    return Scene(means, log_scales, quats, opac, sh)


def mixture_scene(n: int, components: int = 64, sh_degree: int = 3, seed: int = 0,
                  surface_frac: float = 0.3, half_extent: float = 4.0) -> Scene:
    """Scene-scale workload: N Gaussians drawn from an anisotropic mixture.

    Component means are uniform in [-4,4]^3, equal weights, each with covariance
    Q diag(sigma^2) Q^T (sigma log-uniform in [0.1, 1] per axis, Q a random
    rotation).  A fraction ``surface_frac`` of the Gaussians are flattened 'surface'
    Gaussians: one random local axis has log-scale -7.  All other log-scales are
    N(-4, 0.5^2).  Opacity logits N(0,1); SH coefficients N(0, 0.2^2) (DC included).
    """
    rng = np.random.default_rng(seed)
    cm = rng.uniform(-half_extent, half_extent, (components, 3))
    chol = np.empty((components, 3, 3))
    for k in range(components):
        sig = np.exp(rng.uniform(math.log(0.1), math.log(1.0), 3))
        chol[k] = _random_rotation(rng) * sig[None, :]
    comp = rng.integers(0, components, n)
    z = rng.standard_normal((n, 3, 1))
    means = cm[comp] + np.matmul(chol[comp], z)[:, :, 0]
    log_scales = rng.standard_normal((3, n), dtype=np.float32)
    log_scales *= 0.5
    log_scales -= 4.0
    surf = rng.random(n) < surface_frac
    axis = rng.integers(0, 3, n)
    log_scales[axis[surf], np.nonzero(surf)[0]] = -7.0
    quats = _unit_quats(rng, n)
    opac = rng.standard_normal(n, dtype=np.float32)
    k = (sh_degree + 1) ** 2
    sh = rng.standard_normal((k, 3, n), dtype=np.float32)
    sh *= 0.2
    return Scene(np.ascontiguousarray(means.T, dtype=np.float32), log_scales, quats, opac, sh)


def look_at(center, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World-to-camera (R, t) for a camera at ``center`` looking at ``target``
    (x right, y down, z forward)."""
    c = np.asarray(center, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    u = np.asarray(up, dtype=np.float64)
    if abs(np.dot(f, u)) > 0.999:
        u = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, u)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ c
    return R, t


def make_camera(R, t, width: int, height: int, fov_x_deg: float = 60.0, near: float = 0.2,
                fx: float | None = None) -> np.ndarray:
    """One camera record (float32[20]).  fx = W / (2 tan(fov_x/2)), fy = fx (square
    pixels), principal point at the image centre (W-1)/2, (H-1)/2 so that pixel
    centres sit at integer coordinates."""
    if fx is None:
        fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    rec = np.zeros(20, dtype=np.float32)
    rec[0:9] = np.asarray(R, dtype=np.float64).reshape(9)
    rec[9:12] = np.asarray(t, dtype=np.float64)
    rec[12] = fx
    rec[13] = fx
    rec[14] = (width - 1) / 2.0
    rec[15] = (height - 1) / 2.0
    rec[16] = width
    rec[17] = height
    rec[18] = near
    return rec


def cube_corner_cameras(radius: float = 3.0, width: int = 128, height: int = 128,
                        fov_x_deg: float = 60.0) -> np.ndarray:
    """Eight cameras on the cube-corner directions (+-1,+-1,+-1)/sqrt(3) at ``radius``,
    looking at the origin, up = +z."""
    cams = []
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                c = np.array([sx, sy, sz], dtype=np.float64) / math.sqrt(3.0) * radius
                R, t = look_at(c)
                cams.append(make_camera(R, t, width, height, fov_x_deg))
    return np.stack(cams)


def hemisphere_cameras(n_views: int, width: int, height: int, radius: float = 12.0,
                       jitter_deg: float = 5.0, seed: int = 0, fov_x_deg: float = 60.0) -> np.ndarray:
    """``n_views`` cameras on a Fibonacci lattice of the upper hemisphere (z >= 0) at
    ``radius``, each direction jittered by up to +-``jitter_deg`` degrees (seeded),
    looking at the origin, up = +z."""
    rng = np.random.default_rng(seed + 7919)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for k in range(n_views):
        z = 1.0 - (k + 0.5) / n_views  # in (0, 1): upper hemisphere
        rr = math.sqrt(max(0.0, 1.0 - z * z))
        phi = golden * k
        d = np.array([rr * math.cos(phi), rr * math.sin(phi), z])
        j = np.radians(rng.uniform(-jitter_deg, jitter_deg, 2))
        theta = math.acos(max(-1.0, min(1.0, d[2]))) + j[0]
        phi2 = math.atan2(d[1], d[0]) + j[1]
        theta = min(max(theta, 0.0), math.pi / 2)
        d = np.array([math.sin(theta) * math.cos(phi2), math.sin(theta) * math.sin(phi2), math.cos(theta)])
        R, t = look_at(d * radius)
        cams.append(make_camera(R, t, width, height, fov_x_deg))
    return np.stack(cams)


# --- named workloads -------------------------------------------------------------

def workload_small(seed: int = 0):
    """10,000 Gaussians in [-1,1]^3 (SH degree 0) seen by 8 cube-corner cameras at
    128x128 (131,072 pixel-rays); coreset m = 1,000."""
    return uniform_cube_scene(10_000, seed), cube_corner_cameras(3.0, 128, 128), 1000


def workload_scene_1m(seed: int = 0, n_views: int = 100, width: int = 800, height: int = 800):
    """1M Gaussians from a 64-component mixture (SH degree 3), 100 views 800x800."""
    return mixture_scene(1_000_000, 64, 3, seed), hemisphere_cameras(n_views, width, height, seed=seed)


def workload_scene_3m(seed: int = 0, n_views: int = 200, width: int = 1600, height: int = 1040,
                      n: int = 3_000_000):
    """3M Gaussians from a 256-component mixture (SH degree 3), 200 views 1600x1040."""
    return mixture_scene(n, 256, 3, seed), hemisphere_cameras(n_views, width, height, seed=seed)


# (Gaussians, views, width, height) of the six scenes of the batched workload
BATCH6 = ((50_000, 32, 512, 512), (200_000, 64, 800, 600), (500_000, 100, 800, 800),
          (1_000_000, 100, 1024, 768), (2_000_000, 150, 1280, 960), (3_000_000, 200, 1600, 1040))


def workload_batch6(seed: int = 0):
    """Six scenes of uneven size (50k to 3M Gaussians, 64-component mixtures with SH
    degree 3), each with its own hemisphere of 32-200 views at 512x512 to 1600x1040
    (about 7.0e8 pixel-rays in all).  Returns [(scene, cams)]."""
    return [(mixture_scene(n, 64, 3, seed + k), hemisphere_cameras(v, W, H, seed=seed + k))
            for k, (n, v, W, H) in enumerate(BATCH6)]
