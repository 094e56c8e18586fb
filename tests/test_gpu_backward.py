"""The hand-written backward of the weighted-coreset renderer against the FP64 oracle's
analytic gradient (itself pinned by central differences), and the short-recovery
finetune it drives."""
import numpy as np
import pytest

import oracle
from oracle import Opts
import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build, finetune, synth
from parity_helpers import finetune_subcase

pytestmark = pytest.mark.gpu


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


def grad_scene(n=400, seed=0, deg=2):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n), rng.uniform(-0.6, 0.6, n)]).astype(np.float32)
    ls = rng.normal(-3.3, 0.3, (3, n)).astype(np.float32)
    q = rng.standard_normal((4, n))
    q /= np.linalg.norm(q, axis=0)
    op = rng.normal(-0.5, 0.8, n).astype(np.float32)
    sh = (rng.standard_normal(((deg + 1) ** 2, 3, n)) * 0.3).astype(np.float32)
    return synth.Scene(means, ls, q.astype(np.float32), op, sh)


def compare_groups(g_gpu, g_ref, name):
    g_gpu, g_ref = np.asarray(g_gpu, np.float64).ravel(), np.asarray(g_ref, np.float64).ravel()
    err = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    rel = np.abs(g_gpu[big] - g_ref[big]) / np.abs(g_ref[big])
    assert err <= 1e-3, (name, err)
    assert np.quantile(rel, 0.99) <= 1e-3, (name, np.quantile(rel, 0.99))


@pytest.mark.parametrize("weighted", [False, True])
def test_render_backward_matches_oracle(ctx, torch, weighted):
    sc = grad_scene()
    cams = synth.cube_corner_cameras(3.0, 96, 80)[:2]
    sid = ctx.load_scene(sc)
    ctx.set_queries(sid, cams)
    rng = np.random.default_rng(1)
    if weighted:
        idx = np.sort(rng.choice(sc.n, sc.n // 3, replace=False)).astype(np.int32)
        w = rng.uniform(0.5, 2.5, idx.size).astype(np.float32)
        wfull = np.zeros(sc.n)
        wfull[idx] = w
        idx_t, w_t = torch.tensor(idx, device="cuda"), torch.tensor(w, device="cuda")
    else:
        wfull, idx_t, w_t = None, None, None
    for v in range(2):
        r = rng.standard_normal((80, 96, 3)).astype(np.float32)
        gm = torch.zeros(3, sc.n, device="cuda")
        gs = torch.zeros(sc.sh.shape, device="cuda")
        gl = torch.zeros(sc.n, device="cuda")
        ctx.render_backward(sid, v, torch.tensor(r, device="cuda"), gm, gs, gl, idx=idx_t, w=w_t)
        rm, rs, rl = oracle.render_backward(sc, cams[v], r, Opts(), w=wfull)
        compare_groups(gm.cpu().numpy(), rm, "means")
        compare_groups(gs.cpu().numpy(), rs, "sh")
        compare_groups(gl.cpu().numpy(), rl, "opacity_logits")
    ctx.free_scene(sid)


@pytest.mark.parametrize("smooth", [False, True])
def test_backward_on_finetune_subcase_matches_oracle(ctx, torch, smooth):
    """The finetune's gradient sub-case (1,000 SH3 Gaussians with coreset-like weights,
    two 160x104 views): the GPU gradient of <r, weighted render> against the oracle's,
    whose own gradient is pinned by central differences at h = 1e-3 on the same case,
    with the rasteriser's thresholds and without the alpha_min skip at a 7-sigma cut."""
    sc, cams, w = finetune_subcase()
    sid = ctx.load_scene(sc)
    ctx.set_queries(sid, cams)
    idx_t = torch.arange(sc.n, dtype=torch.int32, device="cuda")
    w_t = torch.tensor(w.astype(np.float32), device="cuda")
    w64 = w.astype(np.float32).astype(np.float64)
    # smooth: no alpha_min skip and a 7-sigma footprint; the rho_max = 0.99 clamp stays, since
    # the backward recovers T_i = T_(i+1) / (1 - rho_i) from the back and coreset weights
    # above 1 would otherwise reach rho = 1
    o, go = (Opts(alpha_min=0.0, cut2=49.0), csgs.default_opts(alpha_min=0.0, cut2=49.0)) if smooth \
        else (Opts(), csgs.default_opts())
    rng = np.random.default_rng(24)
    for v in range(2):
        r = rng.standard_normal((104, 160, 3)).astype(np.float32)
        gm = torch.zeros(3, sc.n, device="cuda")
        gs = torch.zeros(sc.sh.shape, device="cuda")
        gl = torch.zeros(sc.n, device="cuda")
        ctx.render_backward(sid, v, torch.tensor(r, device="cuda"), gm, gs, gl, idx=idx_t, w=w_t, opts=go)
        rm, rs, rl = oracle.render_backward(sc, cams[v], r, o, w=w64)
        compare_groups(gm.cpu().numpy(), rm, "means")
        compare_groups(gs.cpu().numpy(), rs, "sh")
        compare_groups(gl.cpu().numpy(), rl, "opacity_logits")
    ctx.free_scene(sid)


def test_finetune_reduces_loss(ctx, torch):
    sc = grad_scene(3000, seed=3, deg=1)
    cams = synth.cube_corner_cameras(3.0, 64, 64)
    sid_full = ctx.load_scene(sc)
    ctx.set_queries(sid_full, cams)
    targets = [ctx.render(sid_full, v, H=64, W=64).clone() for v in range(len(cams))]
    s, S = ctx.score(sid_full)
    idx, w = ctx.sample_coreset(s, 300, 0)
    sub = sc.subset(idx.cpu().numpy())
    sid = ctx.load_scene(sub)
    ctx.set_queries(sid, cams)
    params = {k: torch.tensor(getattr(sub, k), device="cuda").contiguous()
              for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    ar = torch.arange(sub.n, dtype=torch.int32, device="cuda")

    def mean_loss():
        return float(np.mean([float((ctx.render(sid, v, idx=ar, w=w, H=64, W=64) - targets[v]).abs().mean())
                              for v in range(len(cams))]))

    before = mean_loss()
    finetune.finetune(ctx, sid, cams, params, ar, w, targets, steps=60, seed=1)
    after = mean_loss()
    assert after < 0.85 * before, (before, after)
