"""Surrogate-assisted sensitivity scoring (not in the paper).

Exact per-pixel scores (Eq. sen) on a small subset of the query views train the
library's BF16 MLP to predict log-sensitivity; the model is then applied to every
Gaussian with inputs taken over all views, and its prediction is combined with the
exact scores of the scored subset (s = max(exp(prediction) - eps, s_subset)).

Inputs per Gaussian: its attributes, view statistics over all views (views reached,
mean and max projected footprint area) and, with ``lowres_factor`` > 0, the log of a
cheap score: the same per-pixel sensitivity over the scored views and every ``cheap_stride``-th view rendered
at 1/f of the resolution (1/f^2 of the pixel queries).  The cheap score reaches views
the exact scorer skips and carries their occlusion; the network learns, on the scored
views, how the full-resolution score follows from it, from the view statistics and
from the Gaussian's attributes.  With a cheap score (``residual``, the default) the network
predicts the correction of log s over the cheap score scaled by exp(mu), mu the mean
log-ratio of the exact to the cheap score on the scored views: ŝ = max((s_cheap + eps)
exp(mu + prediction) - eps, s_subset), so an output of zero gives the scaled cheap score.
Training rows: the scored views, plus smaller subsets of them (``aug_views``), each with
its statistics and cheap score over the same views and the exact score as the target.

This module only sequences calls into the C ABI (score, view statistics, features,
targets, training, inference, combination); every arithmetic step runs in the
library's kernels.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np


@dataclasses.dataclass
class SurrogateConfig:
    train_views: int = 20          # exact scoring on this many views
    # extra training sets: exact scores of smaller subsets (with the cheap score as an
    # input they cost 1.2 dB on the 3M-Gaussian workload: 17.57 against 18.77 dB at f = 4)
    aug_views: tuple = ()
    eps: float = 1e-8              # target = log(s + eps)
    # 100 steps of 28,416 rows at 5e-3: 19.18 dB in 19.4 ms of training, the same PSNR as 150
    # steps of 56,832 rows at 3e-3 (19.18 dB, 44.5 ms) on the 3M workload
    batch: int = 3 * 148 * 64
    steps: int = 100
    lr: float = 5e-3
    seed: int = 0
    fill_only: bool = False        # use the prediction only where the scored views give s = 0
    # > 0: cheap score at 1/f resolution as an input (0: attributes and view statistics
    # only, which on the 3M workload matched the scored subset alone, 17.00 dB)
    lowres_factor: int = 4
    # cheap score over the scored views and every cheap_stride-th view (its cost is per view:
    # projection and binning of every Gaussian; the scored views' cheap scores are computed
    # for the training rows anyway); 3M workload, 20 scored views, f = 4, pruned-render
    # PSNR, Spearman with the exact scores and total time: every 4th view 19.06 dB, 0.935,
    # 75 ms; every 6th 19.13 dB, 0.923, 67 ms; every 8th 19.00 dB, 0.851, 64 ms; every 12th
    # 19.09 dB, 0.883, 60 ms; exact scoring 18.88 dB in 160 ms
    cheap_stride: int = 6
    # tile shape of the cheap (reduced-resolution) scoring when the caller leaves the shape
    # to the library: 8x8 tiles (a code of the library's TILE_* constants); 34 views of
    # 400 x 260, 3M Gaussians: 15.9 ms against 16.1 (16x8) and 16.9 ms (16x16 tiles)
    cheap_tile_shape: int = 4
    # the network predicts the correction of log s over the cheap score scaled by exp(mu)
    # (mu: the mean log-ratio of the exact to the cheap score on the scored views), so that
    # a zero output reproduces that scaled cheap score; False: it predicts log s itself
    residual: bool = True


def lowres_cameras(cams, f: int) -> np.ndarray:
    """The same cameras at 1/f of the resolution (same field of view): W/f x H/f pixels,
    focal lengths / f, principal point at the centre of the smaller image."""
    cams = np.array(cams, dtype=np.float32).reshape(-1, 20)
    out = cams.copy()
    W = np.maximum(1, cams[:, 16].astype(np.int64) // f)
    H = np.maximum(1, cams[:, 17].astype(np.int64) // f)
    out[:, 12] = cams[:, 12] * (W / cams[:, 16])
    out[:, 13] = cams[:, 13] * (H / cams[:, 17])
    out[:, 14] = (W - 1) / 2.0
    out[:, 15] = (H - 1) / 2.0
    out[:, 16] = W
    out[:, 17] = H
    return out


def view_subset(n_views: int, k: int) -> np.ndarray:
    """k views spread evenly over the query set (indices)."""
    k = max(1, min(k, n_views))
    return np.unique(np.round(np.linspace(0, n_views - 1, k)).astype(int))


def _score_or_zero(ctx, sid, cams, opts):
    """Scores over `cams`, or zeros when every query of them has A = 0."""
    from . import CSGS_E_EMPTY, CsgsError

    ctx.set_queries(sid, cams)
    try:
        s, _ = ctx.score(sid, opts)
    except CsgsError as e:
        if e.status != CSGS_E_EMPTY:
            raise
        s = ctx.torch.zeros(ctx.scene_size(sid), dtype=ctx.torch.float32, device=ctx.device)
    return s.clone()


def _score_into(ctx, sid, opts, out):
    """csgs_score into `out` (with opts.accumulate: the maximum with its contents); a query
    set whose every query has A = 0 leaves it as it is."""
    from . import CSGS_E_EMPTY, CsgsError

    try:
        ctx.score(sid, opts, out=out)
    except CsgsError as e:
        if e.status != CSGS_E_EMPTY:
            raise


def surrogate_scores(ctx, sid: int, cams, cfg: SurrogateConfig | None = None, opts=None, timings: dict | None = None):
    """Returns (s_hat, s_subset) on the device.  Leaves the scene's query set at `cams`."""
    import torch

    from . import TILE_AUTO, default_opts

    cfg = cfg or SurrogateConfig()
    cams = np.asarray(cams, dtype=np.float32).reshape(-1, 20)
    nv = cams.shape[0]
    low = lowres_cameras(cams, cfg.lowres_factor) if cfg.lowres_factor > 0 else None
    opts = opts or default_opts()
    low_opts = opts
    if opts.tile_shape == TILE_AUTO:
        low_opts = copy.copy(opts)
        low_opts.tile_shape = cfg.cheap_tile_shape
    ev = {}

    def mark(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(ctx.stream)
        ev[name] = e

    def rows(views):
        """Features of one training set (statistics and cheap score over `views`), the exact
        score over them and the cheap score (None without one)."""
        s_ex = _score_or_zero(ctx, sid, cams[views], opts)
        s_low = _score_or_zero(ctx, sid, low[views], low_opts) if low is not None else None
        extra = ctx.log_target(s_low, cfg.eps) if s_low is not None else None
        ctx.set_queries(sid, cams[views])
        X = ctx.features(sid, ctx.view_stats(sid, opts), extra)
        return X, s_ex, s_low

    mark("start")
    sub = view_subset(nv, cfg.train_views)
    X0, s_sub, low_sub = rows(sub)
    residual = cfg.residual and low is not None
    mu = ctx.log_ratio_mean(s_sub, low_sub)[0] if residual else 0.0

    def target(s_ex, s_low):
        return ctx.log_residual_target(s_ex, s_low, cfg.eps, mu) if residual else ctx.log_target(s_ex, cfg.eps)

    X_parts, t_parts = [X0], [target(s_sub, low_sub)]
    for k in cfg.aug_views:
        Xk, sk, lk = rows(sub[view_subset(len(sub), k)])
        X_parts.append(Xk)
        t_parts.append(target(sk, lk))
    mark("scored")
    with torch.cuda.stream(ctx.stream):
        X = torch.cat(X_parts)
        t = torch.cat(t_parts)
    ctx.mlp_init(cfg.seed)
    ctx.mlp_train(X, t, batch=cfg.batch, steps=cfg.steps, lr=cfg.lr, seed=cfg.seed + 1)
    mark("trained")
    cheap = None
    if low is not None:
        # the cheap score over the scored views' reduced-resolution copies (already computed
        # for the training rows) and every cheap_stride-th view: s is a maximum over queries
        # (Eq. sen), so the other views are scored into a copy of the first with accumulate
        in_sub = set(int(v) for v in sub)
        extra = [v for v in range(0, nv, max(1, cfg.cheap_stride)) if v not in in_sub]
        cheap = low_sub.clone()
        if extra:
            acc = copy.copy(low_opts)
            acc.accumulate = 1
            ctx.set_queries(sid, low[extra])
            _score_into(ctx, sid, acc, cheap)
    extra = ctx.log_target(cheap, cfg.eps) if cheap is not None else None
    mark("cheap_all")
    ctx.set_queries(sid, cams)
    Xall = ctx.features(sid, ctx.view_stats(sid, opts), extra)
    y = ctx.mlp_forward(Xall)
    s_hat = (ctx.surrogate_combine_prior(y, cheap, s_sub, cfg.eps, mu, cfg.fill_only) if residual
             else ctx.surrogate_combine(y, s_sub, cfg.eps, cfg.fill_only))
    mark("inferred")
    if timings is not None:
        torch.cuda.synchronize()
        timings["exact_subset_ms"] = ev["start"].elapsed_time(ev["scored"])
        timings["train_ms"] = ev["scored"].elapsed_time(ev["trained"])
        timings["cheap_all_views_ms"] = ev["trained"].elapsed_time(ev["cheap_all"])
        timings["infer_ms"] = ev["cheap_all"].elapsed_time(ev["inferred"])
        timings["total_ms"] = ev["start"].elapsed_time(ev["inferred"])
    return s_hat, s_sub


def pruned_psnr(ctx, sid: int, cams, s, m: int, seed: int, views=None, opts=None) -> float:
    """Mean PSNR over views of the weighted coreset (m draws from s) against the full
    render (evaluation metric; colours in [0, 1])."""
    import torch

    cams = np.asarray(cams, dtype=np.float32).reshape(-1, 20)
    views = range(cams.shape[0]) if views is None else views
    idx, w = ctx.sample_coreset(s, m, seed)
    vals = []
    for v in views:
        H, W = int(cams[v][17]), int(cams[v][16])
        full = ctx.render(sid, v, H=H, W=W, opts=opts)
        pr = ctx.render(sid, v, idx=idx, w=w, H=H, W=W, opts=opts)
        mse = float(((full - pr) ** 2).mean())
        vals.append(10.0 * np.log10(1.0 / max(mse, 1e-20)))
    return float(np.mean(vals))
