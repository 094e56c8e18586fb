"""What the trained surrogate adds to exact scoring on a subset of the query views.

Surrogate-assisted scoring scores a few views exactly and fills in the rest with the
trained BF16 network (library kernels only).  Without the network, the subset's scores
are all there is, and every Gaussian that no subset view reaches has probability zero:
it can never enter the coreset.  The test measures, on a seeded scene:
  - coverage: the share of Gaussians with exact s > 0 that get p = 0 without the
    network (positive here) and with it (zero);
  - ranking: the trained network's predictions rank Gaussians by exact sensitivity
    better than an untrained network of the same shape (Spearman 0.18 against 0.00 when
    this was written: a weak but real signal from four scored views);
  - quality: the PSNR of the 90%-pruned render with the subset's scores alone, with the
    surrogate's, and with the exact scores.  These are recorded (in $CSGS_TEST_REPORT_DIR
    when set) and bounded loosely; on these synthetic scenes the surrogate does not beat
    the subset alone in PSNR.
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
    sc = synth.mixture_scene(60000, 32, 3, 5, half_extent=3.0)
    cams = synth.hemisphere_cameras(40, 160, 120, radius=10.0, seed=5)
    sid = ctx.load_scene(sc)
    ctx.set_queries(sid, cams)
    s_ex, _ = ctx.score(sid)
    s_ex = s_ex.clone()
    cfg = surrogate.SurrogateConfig(train_views=4, aug_views=(1, 2), steps=300, fill_only=True)
    s_hat, s_sub = surrogate.surrogate_scores(ctx, sid, cams, cfg)
    a = s_ex.double().cpu().numpy()
    h = s_hat.double().cpu().numpy()
    b = s_sub.double().cpu().numpy()
    pos = a > 0
    lost_without = float(np.mean(b[pos] == 0))
    lost_with = float(np.mean(h[pos] == 0))
    assert lost_without > 0.01  # the subset misses Gaussians other views reach
    assert lost_with == 0.0  # every one of them gets a predicted score

    # trained vs untrained network on the same features (all views)
    X = ctx.features(sid, ctx.view_stats(sid))
    y_trained = ctx.mlp_forward(X).double().cpu().numpy().ravel()
    ctx.mlp_init(123)
    y_untrained = ctx.mlp_forward(X).double().cpu().numpy().ravel()
    r_trained = spearman(a[pos], y_trained[pos])
    r_untrained = spearman(a[pos], y_untrained[pos])
    assert r_trained > r_untrained + 0.1, (r_trained, r_untrained)

    m = int(0.1 * sc.n)
    psnr = {name: surrogate.pruned_psnr(ctx, sid, cams, sv, m, 0, None)
            for name, sv in (("exact", s_ex), ("surrogate", s_hat), ("subset_only", s_sub))}
    report = {"coverage_lost_without": lost_without, "coverage_lost_with": lost_with,
              "spearman_trained": r_trained, "spearman_untrained": r_untrained, "psnr": psnr,
              "gain_psnr_vs_subset": psnr["surrogate"] - psnr["subset_only"],
              "delta_psnr_vs_exact": psnr["surrogate"] - psnr["exact"]}
    out = os.environ.get("CSGS_TEST_REPORT_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "surrogate_gain.json"), "w") as f:
            json.dump(report, f, indent=1)
    assert psnr["surrogate"] > psnr["subset_only"] - 1.0, report
    ctx.free_scene(sid)
