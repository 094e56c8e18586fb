"""Parity at the full 3M-Gaussian, 1600x1040 workload, in the launch configuration the
benchmark times: outputs the oracle can compute one by one (sampled pixels, the exact
sensitivity of chosen Gaussians over a two-view query set) and properties that hold at
any size (1 <= S <= min(N, |Q'|), s <= 1, s_i >= imp(g_i, q) for every sampled q)."""
import numpy as np
import pytest

import oracle
import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

RGB_TOL = 1e-5
S_RTOL = 1e-3


@pytest.fixture(scope="module")
def setup():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    build.build()
    scene, cams = synth.workload_scene_3m()
    ctx = csgs.Context(0)
    sid = ctx.load_scene(scene)
    ctx.set_queries(sid, cams)
    yield scene, cams, oracle.SceneArrays(scene), ctx, sid
    ctx.close()


def test_fullsize_render_sampled_pixels(setup):
    scene, cams, sa, ctx, sid = setup
    rng = np.random.default_rng(1)
    for v in (0, 137):
        rgb = ctx.render(sid, v, H=1040, W=1600).cpu().numpy()
        # sample where the image has content plus uniform pixels
        ys, xs = np.nonzero(rgb.sum(-1) > 0.05)
        pick = rng.choice(len(xs), 96, replace=False)
        pix = np.concatenate([np.stack([xs[pick], ys[pick]], 1), rng.integers(0, [1600, 1040], (32, 2))])
        ref = oracle.render(sa, cams[v], pixels=pix)
        got = rgb[pix[:, 1], pix[:, 0]]
        ok = ~ref["flags"].astype(bool)
        assert ok.mean() >= 0.9
        err = np.abs(got[ok] - ref["rgb"][ok]).max()
        assert err <= RGB_TOL, err


def test_fullsize_score_all_views_bounds(setup):
    scene, cams, sa, ctx, sid = setup
    s, S = ctx.score(sid)
    s = s.cpu().numpy().astype(np.float64)
    st = ctx.stats()
    assert st["views"] == 200 and st["rays"] == 200 * 1600 * 1040
    assert 1.0 <= S <= min(scene.n, st["rays"])
    assert s.max() <= 1.0 + 1e-6 and s.min() >= 0.0
    rng = np.random.default_rng(2)
    for v in (0, 150):
        pix = rng.integers(0, [1600, 1040], (64, 2))
        r = oracle.score_pixels(sa, cams[v], pix)
        lower = np.where(r["touched"], 0.0, r["s"])
        big = lower > 1e-6
        assert np.all(s[big] >= lower[big] * (1 - S_RTOL))


def test_fullsize_exact_sensitivity_two_views(setup):
    scene, cams, sa, ctx, _ = setup
    views = [0, 100]
    sid2 = ctx.load_scene(scene)
    ctx.set_queries(sid2, cams[views])
    s, S = ctx.score(sid2)
    s = s.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    cand = np.nonzero(s > 1e-3)[0]
    chosen = rng.choice(cand, 4, replace=False)
    s_exact = np.zeros(scene.n)
    touched = np.zeros(scene.n, dtype=bool)
    for v in views:
        P = oracle.project(sa, cams[v])
        pix = []
        for g in chosen:
            if P[g, 0] == 0:
                continue
            rx, ry = np.sqrt(9.0 * P[g, 6]) + 1, np.sqrt(9.0 * P[g, 8]) + 1
            x0, x1 = max(0, int(np.ceil(P[g, 1] - rx))), min(1599, int(np.floor(P[g, 1] + rx)))
            y0, y1 = max(0, int(np.ceil(P[g, 2] - ry))), min(1039, int(np.floor(P[g, 2] + ry)))
            for y in range(y0, y1 + 1):
                for x in range(x0, x1 + 1):
                    pix.append((x, y))
        if not pix:
            continue
        r = oracle.score_pixels(sa, cams[v], np.unique(np.array(pix), axis=0))
        s_exact = np.maximum(s_exact, r["s"])
        touched |= r["touched"]
    for g in chosen:
        if touched[g]:
            assert s[g] >= s_exact[g] * (1 - S_RTOL)
        else:
            assert abs(s[g] - s_exact[g]) <= S_RTOL * s_exact[g], (g, s[g], s_exact[g])
    ctx.free_scene(sid2)


def test_fullsize_resolution_chain_and_scene_total(setup):
    """At full size: the per-scene scores sum to 1 (one query, Sec. 3.5), and every
    Gaussian's score can only grow from per-scene to per-image to per-pixel (a max of
    ratios dominates the ratio of sums: the mediant inequality)."""
    scene, cams, sa, ctx, sid = setup
    s_scene, S_scene = ctx.score(sid, csgs.default_opts(resolution=csgs.RES_SCENE))
    assert abs(S_scene - 1.0) < 1e-4
    s_scene = s_scene.cpu().numpy().astype(np.float64)
    s_image = ctx.score(sid, csgs.default_opts(resolution=csgs.RES_IMAGE))[0].cpu().numpy().astype(np.float64)
    s_pixel = ctx.score(sid)[0].cpu().numpy().astype(np.float64)
    tol = 1e-4
    assert np.all(s_image >= s_scene * (1 - tol) - 1e-12)
    assert np.all(s_pixel >= s_image * (1 - tol) - 1e-12)
    assert np.all(s_pixel[s_scene > 0] > 0)  # a Gaussian that contributes anywhere has s > 0
