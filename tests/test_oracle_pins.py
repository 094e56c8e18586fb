"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, published test vectors, library routines, exact
statistics), never against the oracle itself.

The paper prints no worked numeric example (its only numbers are dataset-level
image quality), so the pins are:
  * SH basis: orthonormality on the sphere by Gauss-Legendre quadrature.
  * Philox4x32-10: the published known-answer vectors (tests/golden).
  * Projection: hand-derived closed forms of the EWA covariance for isotropic and
    axis-aligned Gaussians, on and off the optical axis, with a rotated camera.
  * Compositing: closed forms for one and two Gaussians on the optical axis.
  * Scoring: S = 1 for one Gaussian and for the per-scene resolution; 1 <= S <=
    min(N, |Q'|) per pixel; S = N on the isolation scene of Thm. 1; the mediant
    chain s_channel >= s_pixel >= s_tile >= s_image >= s_scene; 1x1 tiles = pixels.
  * Sampling: inverse-CDF draws equal numpy.searchsorted; the uniform map equals
    exact integer arithmetic; frequencies follow p (chi-square); E[w_i] = 1;
    Thm. 2's failure rate is at most delta.
  * Weighted render: w = 1 reproduces the full render bit for bit; the transfer
    sandwich of Lemma "transfer" holds for every pixel.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Opts
from paper_2607_02721_b300 import synth
from parity_helpers import finetune_subcase

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C0 = 1.0 / (2.0 * math.sqrt(math.pi))


def one_scene(means, log_scales, rgb, opac_logit, quats=None):
    """Scene of explicit Gaussians with SH degree 0 colours."""
    means = np.asarray(means, dtype=np.float32).reshape(-1, 3).T.copy()
    n = means.shape[1]
    ls = np.asarray(log_scales, dtype=np.float32).reshape(n, 3).T.copy()
    if quats is None:
        quats = np.tile(np.array([[1.0], [0.0], [0.0], [0.0]], dtype=np.float32), (1, n))
    else:
        quats = np.asarray(quats, dtype=np.float32).reshape(n, 4).T.copy()
    dc = ((np.asarray(rgb, dtype=np.float64).reshape(n, 3) - 0.5) / C0).T.reshape(1, 3, n)
    return synth.Scene(means, ls, quats, np.asarray(opac_logit, dtype=np.float32).reshape(n), dc.astype(np.float32))


def axis_camera(W=33, H=33, f=40.0, R=None, t=(0.0, 0.0, 0.0)):
    R = np.eye(3) if R is None else np.asarray(R)
    return synth.make_camera(R, np.asarray(t), W, H, fx=f)


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-float(np.float32(x))))


def f32(x):
    """The value a float32 input actually carries."""
    return float(np.float32(x))


def eff_scale(sig):
    """Scale carried by the float32 log-scale input."""
    return math.exp(f32(math.log(sig)))


# ---------------------------------------------------------------- SH, Philox

def test_sh_basis_is_orthonormal():
    x, wx = np.polynomial.legendre.leggauss(16)  # exact for polynomials in cos(theta) up to degree 31
    nphi = 32
    phis = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    G = np.zeros((16, 16))
    for ct, wt in zip(x, wx):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = oracle.sh_basis(3, [st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(Y, Y) * wt * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    # the lower degrees are prefixes of the degree-3 basis
    d = np.array([0.3, -0.5, 0.81])
    d /= np.linalg.norm(d)
    Y3 = oracle.sh_basis(3, d)
    for deg in range(3):
        np.testing.assert_array_equal(oracle.sh_basis(deg, d), Y3[: (deg + 1) ** 2])


def _real_sh_from_complex(l, m, d):
    """Real spherical harmonic of degree l, order m along unit vector d, built from
    scipy's complex Y_l^m (which carries the Condon-Shortley phase): sqrt(2) Re Y_l^m
    for m > 0, Y_l^0 for m = 0, sqrt(2) Im Y_l^|m| for m < 0."""
    from scipy.special import sph_harm_y

    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    Y = complex(sph_harm_y(l, abs(m), theta, phi))
    if m == 0:
        return Y.real
    return math.sqrt(2.0) * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_complex_harmonics():
    """Every one of the 16 basis functions (order m = -l..l at index l^2 + l + m), at
    random directions and the six axis directions, against an evaluation that shares
    nothing with the oracle's constants: a sign flip, a swapped order or a wrong
    normalisation of any degree-1..3 function fails here."""
    rng = np.random.default_rng(0)
    dirs = rng.standard_normal((50, 3))
    dirs = np.concatenate([dirs, np.eye(3), -np.eye(3)])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for d in dirs:
        Y = oracle.sh_basis(3, d)
        ref = [_real_sh_from_complex(l, m, d) for l in range(4) for m in range(-l, l + 1)]
        np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-12)


def _sh_scene(mu, coeffs, opac_logit=0.3, sig=0.05):
    """One Gaussian with SH degree 3 colour: ``coeffs`` maps (basis index, channel) to a
    coefficient; every other coefficient is zero."""
    sh = np.zeros((16, 3, 1), dtype=np.float32)
    for (k, ch), v in coeffs.items():
        sh[k, ch, 0] = v
    return synth.Scene(np.asarray(mu, dtype=np.float32).reshape(3, 1),
                       np.full((3, 1), math.log(sig), dtype=np.float32),
                       np.array([[1.0], [0.0], [0.0], [0.0]], dtype=np.float32),
                       np.array([opac_logit], dtype=np.float32), sh)


def test_view_direction_of_the_colour_closed_form():
    """The colour is evaluated along the direction from the camera centre to the mean
    (Sec. 3: view-dependent colour c_i(q)).  A Gaussian at the origin seen along the
    world z axis from below and from above: at the poles the zonal harmonics are
    Y_l^0 = (+-1)^l sqrt((2l + 1) / (4 pi)) (Legendre P_l(+-1) = (+-1)^l), so the
    degree-1 and degree-3 terms change sign between the two cameras and the degree-2
    term does not.  Seen along +x and +y, the order-(+-1) degree-1 functions are
    -sqrt(3 / (4 pi)) x and -sqrt(3 / (4 pi)) y (Condon-Shortley phase).  The centre
    pixel of each render is that colour times the opacity (k = 1 there)."""
    y1 = math.sqrt(3.0 / (4.0 * math.pi))
    y2 = math.sqrt(5.0 / (4.0 * math.pi))
    y3 = math.sqrt(7.0 / (4.0 * math.pi))
    dc = (0.1, -0.2, 0.3)
    coeffs = {(0, 0): dc[0], (0, 1): dc[1], (0, 2): dc[2],
              (2, 0): 0.3, (12, 1): 0.25, (6, 2): 0.2,   # zonal l = 1, 3, 2
              (3, 0): 0.15, (1, 1): -0.35}                # l = 1, m = +1 (x) and m = -1 (y)
    sc = _sh_scene([0.0, 0.0, 0.0], coeffs)
    sh = sc.sh[:, :, 0].astype(np.float64)
    base = C0 * sh[0] + 0.5
    alpha = sigmoid(0.3)
    # camera centres and world-to-camera rotations (rows = camera axes in world
    # coordinates, right-handed), each 2 units from the Gaussian and looking at it
    views = [
        ((0.0, 0.0, -2.0), np.eye(3), (0, 0, 1.0)),
        ((0.0, 0.0, 2.0), np.diag([1.0, -1.0, -1.0]), (0, 0, -1.0)),
        ((-2.0, 0.0, 0.0), np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), (1.0, 0, 0)),
        ((0.0, -2.0, 0.0), np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]), (0, 1.0, 0)),
    ]
    for C, R, d in views:
        assert abs(np.linalg.det(R) - 1.0) < 1e-12
        t = -R @ np.asarray(C)
        cam = axis_camera(W=33, H=33, f=40.0, R=R, t=t)
        x, y, z = d
        expect = base.copy()
        expect[0] += sh[2, 0] * y1 * z + sh[3, 0] * (-y1 * x)
        expect[1] += sh[12, 1] * y3 * z ** 3 + sh[1, 1] * (-y1 * y)
        expect[2] += sh[6, 2] * y2 * (1.5 * z * z - 0.5)
        expect = np.maximum(expect, 0.0)
        P = oracle.project(sc, cam)[0]
        assert P[0] == 1 and abs(P[9] - 2.0) < 1e-12
        np.testing.assert_allclose(P[11:14], expect, rtol=0, atol=1e-12)
        out = oracle.render(sc, cam, Opts())
        np.testing.assert_allclose(out["rgb"][16, 16], expect * alpha, rtol=0, atol=1e-12)
    # the odd degrees really flip: the two z-axis colours differ by 2 y1 c_(l=1) etc.
    P0 = oracle.project(sc, axis_camera(R=views[0][1], t=-views[0][1] @ np.asarray(views[0][0])))[0]
    P1 = oracle.project(sc, axis_camera(R=views[1][1], t=-views[1][1] @ np.asarray(views[1][0])))[0]
    np.testing.assert_allclose(P0[11] - P1[11], 2 * y1 * sh[2, 0], atol=1e-12)
    np.testing.assert_allclose(P0[12] - P1[12], 2 * y3 * sh[12, 1], atol=1e-12)
    np.testing.assert_allclose(P0[13] - P1[13], 0.0, atol=1e-12)


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------------------- projection

DIL = Opts().dilation  # 0.3 as the float32 the options carry


def test_projection_isotropic_on_axis_closed_form():
    sig, z, f, dil = 0.05, 2.0, 40.0, DIL
    sc = one_scene([0, 0, z], [math.log(sig)] * 3, [0.2, 0.5, 0.9], 0.3)
    P = oracle.project(sc, axis_camera(f=f))[0]
    sig = eff_scale(sig)
    var = (f * sig / z) ** 2 + dil
    assert P[0] == 1
    np.testing.assert_allclose(P[1:3], [16.0, 16.0], atol=1e-12)
    np.testing.assert_allclose(P[6:9], [var, 0.0, var], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(P[3:6], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(P[9], z)
    np.testing.assert_allclose(P[10], sigmoid(0.3), rtol=1e-7)
    np.testing.assert_allclose(P[11:14], [0.2, 0.5, 0.9], atol=1e-6)


def test_projection_off_axis_jacobian_closed_form():
    # Sigma = sig^2 I, J = [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]]
    sig, f, dil = 0.07, 50.0, DIL
    x0, y0, z = 0.3, -0.2, 2.5
    sc = one_scene([x0, y0, z], [math.log(sig)] * 3, [0.5, 0.5, 0.5], 0.0)
    P = oracle.project(sc, axis_camera(W=64, H=48, f=f))[0]
    sig, x0, y0 = eff_scale(sig), f32(x0), f32(y0)
    xx = sig * sig * f * f / z / z * (1 + x0 * x0 / z / z) + dil
    yy = sig * sig * f * f / z / z * (1 + y0 * y0 / z / z) + dil
    xy = sig * sig * f * f * x0 * y0 / z ** 4
    np.testing.assert_allclose(P[6:9], [xx, xy, yy], rtol=1e-6)
    np.testing.assert_allclose(P[1:3], [f * x0 / z + 31.5, f * y0 / z + 23.5], rtol=1e-7)


def test_projection_clamps_jacobian_outside_fov():
    # far off-axis: x/z is clamped to 1.3 * (W/2)/f inside J only
    sig, f, dil, W = 0.05, 20.0, DIL, 32
    x0, z = 3.0, 2.0
    sc = one_scene([x0, 0.0, z], [math.log(sig)] * 3, [0.5, 0.5, 0.5], 0.0)
    P = oracle.project(sc, axis_camera(W=W, H=W, f=f))[0]
    sig = eff_scale(sig)
    lim = Opts().clamp_fov * 0.5 * W / f
    assert x0 / z > lim
    xx = sig * sig * f * f / z / z * (1 + lim * lim) + dil
    np.testing.assert_allclose(P[6], xx, rtol=1e-6)
    np.testing.assert_allclose(P[1], f * x0 / z + (W - 1) / 2, rtol=1e-7)


def test_projection_quaternion_and_camera_rotation():
    # 90 degrees about z maps the local x axis to world y: Sigma = diag(sy^2, sx^2, sz^2)
    sx, sy, sz, f, dil, z = 0.02, 0.09, 0.05, 40.0, DIL, 3.0
    q = [math.cos(math.pi / 4), 0.0, 0.0, math.sin(math.pi / 4)]
    sc = one_scene([0, 0, z], [math.log(sx), math.log(sy), math.log(sz)], [0.5] * 3, 0.0, quats=q)
    P = oracle.project(sc, axis_camera(f=f))[0]
    sx, sy, sz = eff_scale(sx), eff_scale(sy), eff_scale(sz)
    k = (f / z) ** 2
    np.testing.assert_allclose(P[6:9], [k * sy * sy + dil, 0.0, k * sx * sx + dil], rtol=1e-6, atol=1e-9)
    # a camera rotated by 90 degrees about world y, placed so the Gaussian is on its axis
    Ry = np.array([[0.0, 0.0, -1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])  # world x -> camera z
    mu = np.array([z, 0.0, 0.0])
    cam = axis_camera(f=f, R=Ry, t=(0.0, 0.0, 0.0))
    sc2 = one_scene(mu, [math.log(sx), math.log(sy), math.log(sz)], [0.5] * 3, 0.0)  # effective values
    P2 = oracle.project(sc2, cam)[0]
    # camera x = -world z, camera y = world y: variances (sz^2, sy^2)
    np.testing.assert_allclose(P2[6:9], [k * sz * sz + dil, 0.0, k * sy * sy + dil], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(P2[9], z)


def test_view_stats_closed_form():
    """Surrogate view statistics of one isotropic Gaussian: two cameras see it on their
    axis at depths 2 and 4 (footprint variance (f sigma / z)^2 + dilation, area
    pi 9 sqrt(det) = 9 pi var), a third looks away from it, a fourth has it far outside
    its image.  A second Gaussian below alpha_min is counted nowhere."""
    sig, f = 0.05, 40.0
    sc = one_scene([[0, 0, 2.0], [0, 0.1, 2.0]], [[math.log(sig)] * 3] * 2, [[0.5] * 3] * 2, [0.3, -9.0])
    R_back = np.diag([1.0, -1.0, -1.0])  # looks along -z from the origin: the Gaussian is behind
    cams = np.stack([axis_camera(f=f), axis_camera(f=f, t=(0.0, 0.0, 2.0)), axis_camera(f=f, R=R_back),
                     axis_camera(f=f, t=(5.0, 0.0, 0.0))])
    st = oracle.view_stats(sc, cams)
    s_eff = eff_scale(sig)
    areas = [9 * math.pi * ((f * s_eff / z) ** 2 + DIL) for z in (2.0, 4.0)]
    np.testing.assert_allclose(st[0], [2, np.mean(areas), max(areas)], rtol=1e-12)
    assert sigmoid(-9.0) < Opts().alpha_min
    np.testing.assert_array_equal(st[1], [0, 0, 0])


# ---------------------------------------------------------------- compositing

def test_single_gaussian_closed_form_render_and_score():
    sig, z, f, dil, lg = 0.04, 2.0, 40.0, DIL, 1.2
    rgb = np.array([0.8, 0.3, 0.6])
    sc = one_scene([0, 0, z], [math.log(sig)] * 3, rgb, lg)
    rgb = C0 * sc.sh[0, :, 0].astype(np.float64) + 0.5
    cam = axis_camera(f=f)
    out = oracle.render(sc, cam, Opts())
    sig = eff_scale(sig)
    var = (f * sig / z) ** 2 + dil
    yy, xx = np.mgrid[0:33, 0:33]
    d2 = ((xx - 16.0) ** 2 + (yy - 16.0) ** 2) / var
    o = Opts()
    rho = np.minimum(o.rho_max, sigmoid(lg) * np.exp(-0.5 * d2))
    rho[(d2 > 9) | (rho < o.alpha_min)] = 0.0
    np.testing.assert_allclose(out["rgb"], rgb[None, None, :] * rho[..., None], atol=1e-6)
    np.testing.assert_allclose(out["T"], 1 - rho, atol=1e-7)
    r = oracle.score(sc, cam[None], Opts())
    np.testing.assert_allclose(r["s"], [1.0], rtol=1e-12)
    assert r["queries"] == int((rho > 0).sum())
    np.testing.assert_allclose(r["S"], 1.0, rtol=1e-12)


def test_two_gaussians_on_axis_closed_form():
    f, dil = 40.0, DIL
    s1, s2, z1, z2, l1, l2 = 0.03, 0.06, 1.5, 2.5, 0.4, -0.2
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.7, 0.6])
    sc = one_scene([[0, 0, z2], [0, 0, z1]], [[math.log(s2)] * 3, [math.log(s1)] * 3], [c2, c1], [l2, l1])
    c2, c1 = (C0 * sc.sh[0, :, 0].astype(np.float64) + 0.5), (C0 * sc.sh[0, :, 1].astype(np.float64) + 0.5)
    cam = axis_camera(f=f)
    yy, xx = np.mgrid[0:33, 0:33]
    r2 = (xx - 16.0) ** 2 + (yy - 16.0) ** 2

    def rho(s, z, lg):
        v = (f * eff_scale(s) / z) ** 2 + dil
        o = Opts()
        r = np.minimum(o.rho_max, sigmoid(lg) * np.exp(-0.5 * r2 / v))
        r[(r2 / v > 9) | (r < o.alpha_min)] = 0.0
        return r

    p1, p2 = rho(s1, z1, l1), rho(s2, z2, l2)  # Gaussian index 1 is in front
    A = c1[None, None] * p1[..., None] + c2[None, None] * (p2 * (1 - p1))[..., None]
    out = oracle.render(sc, cam, Opts())
    np.testing.assert_allclose(out["rgb"], A, atol=1e-12)
    np.testing.assert_allclose(out["T"], (1 - p1) * (1 - p2), atol=1e-12)
    a1 = c1.sum() * p1
    a2 = c2.sum() * p2 * (1 - p1)
    At = a1 + a2
    m = At > 0
    s_expect = [np.max(a2[m] / At[m]), np.max(a1[m] / At[m])]
    r = oracle.score(sc, cam[None], Opts())
    np.testing.assert_allclose(r["s"], s_expect, rtol=1e-12)
    # luminance objective of the per-pixel resolution
    wl = (0.299, 0.587, 0.114)
    a1l, a2l = np.dot(c1, wl) * p1, np.dot(c2, wl) * p2 * (1 - p1)
    rl = oracle.score(sc, cam[None], Opts(obj_w=wl))
    np.testing.assert_allclose(rl["s"], [np.max(a2l[m] / (a1l + a2l)[m]), np.max(a1l[m] / (a1l + a2l)[m])], rtol=1e-12)


def test_two_gaussians_resolutions_and_variants_closed_form():
    """Sec. 3.5's resolutions and variants written out by hand for two Gaussians on
    the optical axis (index 1 in front), from the per-pixel closed forms
    rho_1, rho_2, T_1 = 1, T_2 = 1 - rho_1:
      channel  s_i = max over (pixel, lambda) with A_lambda > 0 of a_i,lambda / A_lambda
      tile     s_i = max over 11x11 tiles of (sum_tile a_i) / (sum_tile A)
      image    s_i = (sum_image a_i) / (sum_image A)  (one view: the scene query)
      L2       a_i = sum_lambda (c_i,lambda rho_i T_i)^2,  no-colour  a_i = rho_i T_i
    with A the sum of the same terms over the pixel's contributors."""
    f, dil = 40.0, DIL
    s1, s2, z1, z2, l1, l2 = 0.03, 0.06, 1.5, 2.5, 0.4, -0.2
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.7, 0.6])
    sc = one_scene([[0, 0, z2], [0, 0, z1]], [[math.log(s2)] * 3, [math.log(s1)] * 3], [c2, c1], [l2, l1])
    c2, c1 = (C0 * sc.sh[0, :, 0].astype(np.float64) + 0.5), (C0 * sc.sh[0, :, 1].astype(np.float64) + 0.5)
    cam = axis_camera(f=f)
    yy, xx = np.mgrid[0:33, 0:33]
    r2 = (xx - 16.0) ** 2 + (yy - 16.0) ** 2
    o = Opts()

    def rho(s, z, lg):
        v = (f * eff_scale(s) / z) ** 2 + dil
        r = np.minimum(o.rho_max, sigmoid(lg) * np.exp(-0.5 * r2 / v))
        r[(r2 / v > 9) | (r < o.alpha_min)] = 0.0
        return r

    p1, p2 = rho(s1, z1, l1), rho(s2, z2, l2)
    w1, w2 = p1, p2 * (1 - p1)                      # rho T of each contributor
    a1c, a2c = c1 * w1[..., None], c2 * w2[..., None]  # per-channel L1 terms [33, 33, 3]

    def score(**kw):
        return oracle.score(sc, cam[None], Opts(**kw))["s"]  # [Gaussian 0 (back), 1 (front)]

    # per-channel (L1)
    A = a1c + a2c
    m = A > 0
    np.testing.assert_allclose(score(resolution=oracle.RES_CHANNEL),
                               [np.max(a2c[m] / A[m]), np.max(a1c[m] / A[m])], rtol=1e-12)
    # per-pixel L2 and no-colour
    for var, t1, t2 in ((oracle.VAR_L2, (a1c ** 2).sum(-1), (a2c ** 2).sum(-1)), (oracle.VAR_NC, w1, w2)):
        At = t1 + t2
        mm = At > 0
        np.testing.assert_allclose(score(variant=var), [np.max(t2[mm] / At[mm]), np.max(t1[mm] / At[mm])],
                                   rtol=1e-12)
    # per-channel L2: each channel's own squared terms
    A2 = a1c ** 2 + a2c ** 2
    m2 = A2 > 0
    np.testing.assert_allclose(score(resolution=oracle.RES_CHANNEL, variant=oracle.VAR_L2),
                               [np.max(a2c[m2] ** 2 / A2[m2]), np.max(a1c[m2] ** 2 / A2[m2])], rtol=1e-12)
    # per-tile (11x11 tiles of the 33x33 image) and per-image, L1 pixel objective
    t1, t2 = a1c.sum(-1), a2c.sum(-1)
    tiles = []
    for ty in range(3):
        for tx in range(3):
            sl = (slice(11 * ty, 11 * ty + 11), slice(11 * tx, 11 * tx + 11))
            At = t1[sl].sum() + t2[sl].sum()
            if At > 0:
                tiles.append((t2[sl].sum() / At, t1[sl].sum() / At))
    np.testing.assert_allclose(score(resolution=oracle.RES_TILE, tile=11), np.max(np.array(tiles), 0), rtol=1e-12)
    Ai = t1.sum() + t2.sum()
    np.testing.assert_allclose(score(resolution=oracle.RES_IMAGE), [t2.sum() / Ai, t1.sum() / Ai], rtol=1e-12)
    np.testing.assert_allclose(score(resolution=oracle.RES_SCENE), [t2.sum() / Ai, t1.sum() / Ai], rtol=1e-12)


def test_early_termination_and_order_invariants():
    sc = synth.uniform_cube_scene(300, seed=3)
    cam = synth.cube_corner_cameras(3.0, 40, 40)[0]
    o = Opts()
    out = oracle.render(sc, cam, o)
    assert np.all(out["T"] >= o.t_min)
    P = oracle.project(sc, cam, o)
    for (px, py) in [(20, 20), (10, 25), (31, 7), (0, 0)]:
        t = oracle.pixel_terms(sc, cam, px, py, o)
        if len(t["gid"]) == 0:
            continue
        d = P[t["gid"], 9]
        assert np.all(np.diff(d) >= 0)
        assert np.all((t["rho"] >= o.alpha_min) & (t["rho"] <= o.rho_max))
        np.testing.assert_allclose(t["T"], np.concatenate([[1.0], np.cumprod(1 - t["rho"])[:-1]]), rtol=1e-13)
        np.testing.assert_allclose((t["rgb"] * (t["rho"] * t["T"])[:, None]).sum(0), out["rgb"][py, px], rtol=1e-12)
        np.testing.assert_allclose(t["T"][-1] * (1 - t["rho"][-1]), out["T"][py, px], rtol=1e-12)


# ---------------------------------------------------------------- scoring

def small_scene(n=400, seed=1):
    return synth.uniform_cube_scene(n, seed=seed), synth.cube_corner_cameras(3.0, 32, 32)[:3]


def test_sensitivity_bounds_per_pixel():
    sc, cams = small_scene()
    r = oracle.score(sc, cams, Opts())
    assert r["queries"] > 0
    assert 1.0 - 1e-12 <= r["S"] <= min(sc.n, r["queries"]) + 1e-9
    assert np.all(r["s"] <= 1.0 + 1e-15) and np.all(r["s"] >= 0)


def test_scene_resolution_total_sensitivity_is_one():
    sc, cams = small_scene()
    r = oracle.score(sc, cams, Opts(resolution=oracle.RES_SCENE))
    np.testing.assert_allclose(r["S"], 1.0, rtol=1e-12)


def test_resolution_mediant_chain():
    sc, cams = small_scene(300, seed=5)
    s = {}
    for name, res in [("channel", oracle.RES_CHANNEL), ("pixel", oracle.RES_PIXEL), ("tile", oracle.RES_TILE),
                      ("image", oracle.RES_IMAGE), ("scene", oracle.RES_SCENE)]:
        s[name] = oracle.score(sc, cams, Opts(resolution=res, tile=8))["s"]
    tol = 1e-12
    assert np.all(s["channel"] >= s["pixel"] - tol)
    assert np.all(s["pixel"] >= s["tile"] - tol)
    assert np.all(s["tile"] >= s["image"] - tol)
    assert np.all(s["image"] >= s["scene"] - tol)
    # 1x1 tiles are pixels
    s1 = oracle.score(sc, cams, Opts(resolution=oracle.RES_TILE, tile=1))["s"]
    np.testing.assert_allclose(s1, s["pixel"], rtol=1e-12, atol=1e-300)
    # one view: the image query is the scene query
    np.testing.assert_allclose(oracle.score(sc, cams[:1], Opts(resolution=oracle.RES_IMAGE))["s"],
                               oracle.score(sc, cams[:1], Opts(resolution=oracle.RES_SCENE))["s"], rtol=1e-10)


def test_score_variants_definitions():
    # no-colour: A^nc per pixel equals 1 - T_final under the pure definitions
    sc, cams = small_scene(200, seed=9)
    o = Opts.pure(variant=oracle.VAR_NC)
    cam = cams[0]
    out = oracle.render(sc, cam, o)
    for (px, py) in [(16, 16), (5, 20)]:
        t = oracle.pixel_terms(sc, cam, px, py, o)
        np.testing.assert_allclose((t["rho"] * t["T"]).sum(), 1 - out["T"][py, px], rtol=1e-12)
    # the L2 variant never exceeds the bounds either
    r = oracle.score(sc, cams, Opts(variant=oracle.VAR_L2))
    assert 1 - 1e-12 <= r["S"] <= min(sc.n, r["queries"]) + 1e-9


def test_isolation_scene_theorem1():
    # N far-apart tiny Gaussians; camera i sits right in front of Gaussian i, so at
    # its centre pixel Gaussian i is the only contributor: s_i = 1 and S = N.
    n = 6
    means = [[10.0 * i, 0.0, 0.0] for i in range(n)]
    sc = one_scene(means, [[math.log(0.01)] * 3] * n, [[0.6, 0.4, 0.3]] * n, [0.5] * n)
    cams = []
    for i in range(n):
        R, t = synth.look_at([10.0 * i, -1.0, 0.0], target=[10.0 * i, 0.0, 0.0])
        cams.append(synth.make_camera(R, t, 5, 5, fx=20.0))
    r = oracle.score(sc, np.stack(cams), Opts())
    np.testing.assert_allclose(r["s"], np.ones(n), rtol=1e-12)
    np.testing.assert_allclose(r["S"], n, rtol=1e-12)


# ---------------------------------------------------------------- sampling

def test_uniform_map_and_inverse_cdf_against_integer_math_and_searchsorted():
    rng = np.random.default_rng(0)
    s = rng.random(257) ** 3
    s[rng.random(257) < 0.2] = 0.0
    p, S = oracle.probabilities(s)
    np.testing.assert_allclose(S, s.sum(), rtol=1e-15)
    C = oracle.cdf(p)
    total = int(C[-1])
    assert abs(total - 2 ** 56) <= len(p)
    assert np.all(np.diff(C.astype(object)) >= 0)
    seed, m = 1234567, 500
    r = oracle.sample(p, m, seed)
    for t in range(m):
        ctr = [t & 0xFFFFFFFF, t >> 32, 0, 0]
        w = oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        x = (int(w[1]) << 32) | int(w[0])
        u = (x * total) >> 64
        assert u == oracle.uniform(seed, t, total)
        j = int(np.searchsorted(C.astype(object), u, side="right"))
        assert r["J"][t] == j
        assert p[j] > 0
    assert r["counts"].sum() == m
    assert r["distinct"] == len(r["idx"]) <= m
    np.testing.assert_allclose(r["w_sel"], r["counts"][r["idx"]] / (m * p[r["idx"]]), rtol=1e-15)


def test_sample_frequencies_follow_p():
    rng = np.random.default_rng(1)
    p = rng.random(40)
    p /= p.sum()
    m = 200_000
    r = oracle.sample(p, m, 99)
    expected = m * p
    chi2 = ((r["counts"] - expected) ** 2 / expected).sum()
    # 39 degrees of freedom: P(chi2 > 80) < 1e-4
    assert chi2 < 80.0


def test_weights_are_unbiased():
    rng = np.random.default_rng(2)
    p = rng.random(30) + 0.05
    p /= p.sum()
    m, seeds = 20, 3000
    W = np.stack([oracle.sample(p, m, 1000 + k)["w"] for k in range(seeds)])
    mean = W.mean(0)
    se = W.std(0) / math.sqrt(seeds)
    assert np.all(np.abs(mean - 1.0) <= 4.5 * se + 1e-12)


def test_theorem2_failure_rate_at_most_delta():
    sc, cams = small_scene(150, seed=4)
    o = Opts.pure()
    r = oracle.score(sc, cams, o)
    p, S = oracle.probabilities(r["s"])
    eps, delta = 0.5, 0.25
    m = int(math.ceil(oracle.theorem2_m(S, eps, delta, r["queries"])))
    assert m == int(math.ceil(3 * S / eps ** 2 * math.log(2 * r["queries"] / delta)))
    fails, trials = 0, 24
    for k in range(trials):
        w = oracle.sample(p, m, 77 + k)["w"]
        worst = 0.0
        for cam in cams:
            t = oracle.transfer(sc, cam, w, o)
            A = t["A"].sum(-1)
            Ath = t["A_th"].sum(-1)
            msk = A > 0
            worst = max(worst, float(np.max(np.abs(Ath[msk] - A[msk]) / A[msk])))
        fails += worst > eps
    assert fails / trials <= delta


# ---------------------------------------------------------------- weighted render

def test_unit_weights_reproduce_full_render():
    sc, cams = small_scene(300, seed=6)
    a = oracle.render(sc, cams[1], Opts())
    b = oracle.render(sc, cams[1], Opts(), w=np.ones(sc.n))
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    np.testing.assert_array_equal(a["T"], b["T"])
    assert b["violations"] == 0


def test_transfer_sandwich_and_weighted_render_agree():
    sc, cams = small_scene(300, seed=8)
    o = Opts.pure()
    r = oracle.score(sc, cams, o)
    p, S = oracle.probabilities(r["s"])
    w = oracle.sample(p, 120, 5)["w"]
    for cam in cams:
        t = oracle.transfer(sc, cam, w, o)
        valid = t["min_factor"] > 0
        g = t["gamma"][..., None]
        lo = np.exp(-g) * t["A_th"]
        hi = np.exp(g) * t["A_th"]
        ok = (t["A_w"] >= lo * (1 - 1e-12) - 1e-15) & (t["A_w"] <= hi * (1 + 1e-12) + 1e-15)
        assert np.all(ok[valid])
        # the same reduced render through the renderer with weights (alpha' = w alpha)
        rw = oracle.render(sc, cam, o, w=w)
        np.testing.assert_allclose(rw["rgb"][valid], t["A_w"][valid], rtol=1e-10, atol=1e-14)
        rf = oracle.render(sc, cam, o)
        np.testing.assert_allclose(rf["rgb"], t["A"], rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- surrogate MLP

def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to even (1)
    assert oracle.bf16(1.0 + 2 ** -8) == 1.0
    assert oracle.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert oracle.bf16(1.0 + 2 ** -8 + 2 ** -12) == 1.0 + 2 ** -7
    assert oracle.bf16(-3.0) == -3.0 and oracle.bf16(0.0) == 0.0
    # against torch's bfloat16 conversion (a library routine)
    import torch
    x = torch.randn(2000, dtype=torch.float32) * 10
    ref = x.to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16(float(v)) for v in x])
    np.testing.assert_array_equal(got, ref)


def test_gelu_and_derivative():
    from math import erf, sqrt, exp, pi
    for z in (-3.0, -0.7, 0.0, 0.3, 2.5):
        assert oracle.gelu(z) == pytest.approx(0.5 * z * (1 + erf(z / sqrt(2))), rel=1e-15, abs=1e-300)
        h = 1e-6
        fd = (oracle.gelu(z + h) - oracle.gelu(z - h)) / (2 * h)
        assert oracle.gelu_d(z) == pytest.approx(fd, rel=1e-8, abs=1e-10)
    assert oracle.gelu(0.0) == 0.0 and oracle.gelu_d(0.0) == 0.5


def _mlp_params(seed=0, scale=0.15):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(oracle.mlp_nparam()) * scale


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    P = _mlp_params(2)
    X = rng.standard_normal((6, oracle.MLP_IN)).astype(np.float32)
    t = rng.standard_normal(6).astype(np.float32)
    loss, G = oracle.mlp_backward(P, X, t, emulate=False)
    idx = np.concatenate([rng.choice(oracle.MLP_H * oracle.MLP_IN, 12, replace=False),
                          oracle.MLP_H * oracle.MLP_IN + rng.choice(oracle.mlp_nparam() - oracle.MLP_H * oracle.MLP_IN, 20,
                                                                    replace=False)])
    h = 1e-3
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        lp = np.mean((oracle.mlp_forward(Pp, X, emulate=False) - t) ** 2)
        lm = np.mean((oracle.mlp_forward(Pm, X, emulate=False) - t) ** 2)
        fd = (lp - lm) / (2 * h)
        assert G[i] == pytest.approx(fd, rel=2e-4, abs=1e-8)
    assert loss == pytest.approx(np.mean((oracle.mlp_forward(P, X, emulate=False) - t) ** 2), rel=1e-14)


def test_mlp_forward_matches_a_dense_reference():
    # the network written with numpy matrix products (a library routine) and erf
    from math import erf, sqrt
    rng = np.random.default_rng(3)
    P = _mlp_params(4)
    X = rng.standard_normal((5, oracle.MLP_IN)).astype(np.float32)
    W1, b1, W2, b2, w3, b3 = oracle.mlp_split(P)
    g = np.vectorize(lambda z: 0.5 * z * (1 + erf(z / sqrt(2))))
    y = g(g(X.astype(np.float64) @ W1.T + b1) @ W2.T + b2) @ w3 + b3[0]
    np.testing.assert_allclose(oracle.mlp_forward(P, X, emulate=False), y, rtol=1e-12)


def test_adam_first_step_moves_by_lr():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-4, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(p, g, m, v, 1e-2, 1)
    # bias-corrected first step: -lr * g / (|g| + eps)
    np.testing.assert_allclose(p, [1.0 - 1e-2 * 0.3 / (0.3 + 1e-8), -2.0 + 1e-2 * 1e-4 / (1e-4 + 1e-8), 0.5], rtol=1e-12)


# ---------------------------------------------------------------- render gradient

def _grad_scene(n=10, seed=0, deg=2):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.35, 0.35, n), rng.uniform(-0.35, 0.35, n), rng.uniform(1.5, 3.0, n)]).astype(np.float32)
    ls = rng.uniform(-3.2, -2.2, (3, n)).astype(np.float32)
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0)
    op = rng.normal(-0.5, 0.8, n).astype(np.float32)
    sh = (rng.standard_normal(((deg + 1) ** 2, 3, n)) * 0.3).astype(np.float32)
    return synth.Scene(means, ls, q.astype(np.float32), op, sh)


def test_render_gradient_matches_central_differences():
    sc = _grad_scene()
    cam = axis_camera(W=24, H=20, f=30.0)
    o = Opts.pure(cut2=1e4)  # smooth: no footprint cut, no thresholds
    rng = np.random.default_rng(1)
    r = rng.standard_normal((20, 24, 3))
    w = rng.uniform(0.5, 1.5, sc.n)
    gm, gs, gl = oracle.render_backward(sc, cam, r, o, w=w)

    def L(s):
        return float((oracle.render(s, cam, o, w=w)["rgb"] * r).sum())

    h = 1e-4
    checks = 0
    for arr_name, grad in (("means", gm), ("sh", gs), ("opacity_logits", gl)):
        arr = getattr(sc, arr_name)
        flat_idx = rng.choice(arr.size, min(12, arr.size), replace=False)
        for fi in flat_idx:
            ix = np.unravel_index(fi, arr.shape)
            base = arr[ix]
            vals = []
            for sgn in (1, -1):
                s2 = synth.Scene(sc.means.copy(), sc.log_scales, sc.quats, sc.opacity_logits.copy(), sc.sh.copy())
                a2 = getattr(s2, arr_name)
                a2[ix] = np.float32(float(base) + sgn * h)
                vals.append((L(s2), float(a2[ix]) - float(base)))
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert grad[ix] == pytest.approx(fd, rel=2e-3, abs=2e-4), (arr_name, ix, grad[ix], fd)
            checks += 1
    assert checks == 34


def test_render_gradient_central_differences_on_finetune_subcase():
    """Oracle gradient of L = sum over the two views of <r_v, weighted render_v> against
    central differences with h = 1e-3 (the benchmark's stated step), on the smooth
    definitions (alpha_min = 0, rho_max = 1, t_min = 0, footprint cut at 7 sigma, where the
    kernel is below 3e-11).  A mean whose perturbation changes its depth rank in a view
    (a change of the compositing order, where L is not differentiable) is skipped."""
    sc, cams, w = finetune_subcase()
    o = Opts.pure(cut2=49.0)
    rng = np.random.default_rng(23)
    rs = [rng.standard_normal((104, 160, 3)) for _ in cams]
    grads = [oracle.render_backward(sc, cam, r, o, w=w) for cam, r in zip(cams, rs)]
    g = [sum(gv[k] for gv in grads) for k in range(3)]

    def L(s):
        return sum(float((oracle.render(s, cam, o, w=w)["rgb"] * r).sum()) for cam, r in zip(cams, rs))

    def rank(s, i):
        return [int(np.sum(oracle.project(s, cam, o)[:, 9] < oracle.project(s, cam, o)[i, 9])) for cam in cams]

    h = 1e-3
    checks = 0
    for arr_name, grad in (("means", g[0]), ("sh", g[1]), ("opacity_logits", g[2])):
        arr = getattr(sc, arr_name)
        big = np.flatnonzero(np.abs(grad).ravel() > 1e-2 * np.abs(grad).max())
        for fi in rng.choice(big, 8, replace=False):
            ix = np.unravel_index(fi, arr.shape)
            base = arr[ix]
            vals, ranks = [], []
            for sgn in (1, -1):
                s2 = synth.Scene(sc.means.copy(), sc.log_scales, sc.quats, sc.opacity_logits.copy(), sc.sh.copy())
                a2 = getattr(s2, arr_name)
                a2[ix] = np.float32(float(base) + sgn * h)
                vals.append((L(s2), float(a2[ix]) - float(base)))
                if arr_name == "means":
                    ranks.append(rank(s2, ix[1]))
            if ranks and ranks[0] != ranks[1]:
                continue
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert grad[ix] == pytest.approx(fd, rel=5e-3, abs=1e-9), (arr_name, ix, grad[ix], fd)
            checks += 1
    assert checks >= 20


def test_render_gradient_of_unit_weight_scene_matches_unweighted():
    sc = _grad_scene(8, seed=2, deg=1)
    cam = axis_camera(W=16, H=16, f=24.0)
    r = np.random.default_rng(3).standard_normal((16, 16, 3))
    a = oracle.render_backward(sc, cam, r, Opts())
    b = oracle.render_backward(sc, cam, r, Opts(), w=np.ones(sc.n))
    for x, y in zip(a, b):  # equal up to the order of the parallel accumulation
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-15)


def test_tiled_traversal_equals_brute_force():
    """The rasteriser's traversal (per-tile lists from the footprint boxes) gives exactly
    the brute-force render, for the standard 16x16 tiles, the GPU's, and odd shapes, with
    and without coreset weights: tiling loses nothing (the footprint test is per pixel)."""
    sc, _ = small_scene()
    cams = synth.cube_corner_cameras(3.0, 48, 40)
    w = np.random.default_rng(3).uniform(0.5, 3.0, sc.n)
    for cam in cams[:3]:
        for weights in (None, w):
            ref = oracle.render(sc, cam, w=weights)
            for tw, th in ((16, 16), (32, 16), (7, 5), (64, 64)):
                t = oracle.render_tiled(sc, cam, tw, th, w=weights)
                assert np.array_equal(t["rgb"], ref["rgb"]), (tw, th)
                assert np.array_equal(t["T"], ref["T"]) and np.array_equal(t["n_terms"], ref["n_terms"])
