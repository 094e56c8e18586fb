"""What the trained surrogate adds to exact scoring on a subset of the query views, on a
small seeded scene (the 3M-Gaussian workload's target is checked in test_gpu_fullsize).

Surrogate-assisted scoring scores 10% of the views exactly at full resolution and
predicts every Gaussian's per-pixel sensitivity over all views with the library's BF16
network, from its attributes, view statistics over all views and a cheap score: the same
per-pixel sensitivity over every 4th view rendered at a quarter of the resolution.  The
network is trained on the scored views only.  The test asserts that no Gaussian with
exact s > 0 gets p = 0 (without the network a few percent do) and that the 90%-pruned
render (PSNR against the full render) beats the scored subset's exact scores alone.  It
records, without asserting, the exact scores' PSNR and an un-learned combination of the
same inputs (the cheap score scaled to the exact scores by the median ratio on the scored
views, maximum with the subset's scores).  Written to
$CSGS_TEST_REPORT_DIR/surrogate_gain.json when set.
"""
import json
import os

import numpy as np
import pytest

import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build, surrogate, synth

pytestmark = pytest.mark.gpu


def spearman(a, b):
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    return float(np.corrcoef(ra, rb)[0, 1])


@pytest.fixture(scope="module")
def torch():
    import torch as t

    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    build.build()
    c = csgs.Context(0)
    yield c
    c.close()


def test_surrogate_gain_over_subset_scores(ctx, torch):
    sc = synth.mixture_scene(300_000, 64, 3, 5, half_extent=3.5)
    cams = synth.hemisphere_cameras(40, 640, 416, radius=10.0, seed=5)
    sid = ctx.load_scene(sc)
    ctx.set_queries(sid, cams)
    s_ex, _ = ctx.score(sid)
    s_ex = s_ex.clone()
    cfg = surrogate.SurrogateConfig(train_views=4, cheap_stride=4)
    s_hat, s_sub = surrogate.surrogate_scores(ctx, sid, cams, cfg)
    a = s_ex.double().cpu().numpy()
    h = s_hat.double().cpu().numpy()
    b = s_sub.double().cpu().numpy()
    pos = a > 0
    lost_without = float(np.mean(b[pos] == 0))
    lost_with = float(np.mean(h[pos] == 0))
    # the cheap score alone, brought to the exact scale by the median ratio on the scored
    # views and combined with the subset's exact scores (no network)
    low = surrogate.lowres_cameras(cams, cfg.lowres_factor)
    ctx.set_queries(sid, low[::cfg.cheap_stride])
    s_low = ctx.score(sid)[0].clone()
    sub = surrogate.view_subset(len(cams), cfg.train_views)
    ctx.set_queries(sid, low[sub])
    s_low_sub = ctx.score(sid)[0].double().cpu().numpy()
    ok = (b > 0) & (s_low_sub > 0)
    ratio = float(np.median(b[ok] / s_low_sub[ok]))
    s_nonet = torch.maximum(s_sub, s_low * ratio)
    ctx.set_queries(sid, cams)
    m = int(0.1 * sc.n)
    psnr = {name: surrogate.pruned_psnr(ctx, sid, cams, sv, m, 0, None)
            for name, sv in (("exact", s_ex), ("surrogate", s_hat), ("subset_only", s_sub), ("no_network", s_nonet))}
    report = {"coverage_lost_without": lost_without, "coverage_lost_with": lost_with,
              "spearman_surrogate": spearman(a[pos], h[pos]),
              "spearman_no_network": spearman(a[pos], s_nonet.double().cpu().numpy()[pos]), "psnr": psnr,
              "gain_psnr_vs_subset": psnr["surrogate"] - psnr["subset_only"],
              "delta_psnr_vs_exact": psnr["surrogate"] - psnr["exact"]}
    out = os.environ.get("CSGS_TEST_REPORT_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "surrogate_gain.json"), "w") as f:
            json.dump(report, f, indent=1)
    assert lost_without > 0.01, report
    assert lost_with == 0.0, report
    assert psnr["surrogate"] > psnr["subset_only"], report
    ctx.free_scene(sid)
