"""View-sharded sensitivity scoring over several GPUs, one process per GPU.

The query set of Algorithm 1 is the union of the views' pixel queries, and every query
resolution of Sec. 3.5 combines over views by an associative operation:
  - per-pixel, per-channel, per-tile and per-image sensitivities are maxima over
    queries (Eq. sen), so the maximum over ranks of each rank's scores over its own
    views is the score over all views, bit for bit;
  - the per-scene sensitivity is a ratio of sums over queries, s = sum_q a / sum_q A:
    a rank's scores s_r over its views, scaled by its share A_r / A of the objective
    total, summed over ranks, give the score over all views.
One collective per scoring call (all-reduce MAX of N floats, or SUM of one double and N
floats) is the only exchange; sampling needs none, because every rank draws the same
coreset from the same scores and seed (counter-based uniforms).

This module only partitions the views and sequences the library's calls and the
collective; every per-Gaussian arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

RES_SCENE = 1


def shard_views(n_views: int, rank: int, world: int) -> np.ndarray:
    """Views of rank ``rank``: v = rank, rank + world, ... (round-robin, so every rank
    gets views from all parts of the camera rig)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return np.arange(rank, n_views, world, dtype=np.int64)


def combine_shards(s_local, objective_local: float, resolution: int, dist, scale, group=None):
    """Combine this rank's scores over its views with the other ranks' (in place).

    s_local: float32 tensor [N] (on the device the process group's backend uses);
    objective_local: this rank's sum of A(q) over its queries (per-scene resolution only);
    scale(tensor, factor): multiplies the tensor by factor in place (the library's kernel).
    Returns s_local, now the scores over every rank's views."""
    if resolution == RES_SCENE:
        import torch

        tot = torch.tensor([float(objective_local)], dtype=torch.float64, device=s_local.device)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM, group=group)
        total = float(tot.item())
        scale(s_local, objective_local / total if total > 0.0 else 0.0)
        dist.all_reduce(s_local, op=dist.ReduceOp.SUM, group=group)
    else:
        dist.all_reduce(s_local, op=dist.ReduceOp.MAX, group=group)
    return s_local


def sharded_score(ctx, sid: int, cams, opts, dist, group=None, out=None):
    """Scores of the whole query set ``cams`` with this rank scoring its round-robin share
    of the views; returns (s, S), identical on every rank.  Leaves the scene's query set
    at this rank's views."""
    from . import CSGS_E_EMPTY, CsgsError

    cams = np.asarray(cams, dtype=np.float32).reshape(-1, 20)
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    views = shard_views(cams.shape[0], rank, world)
    n = ctx.scene_size(sid)
    torch = ctx.torch
    s = out if out is not None else torch.empty(n, dtype=torch.float32, device=ctx.device)
    objective = 0.0
    if len(views):
        ctx.set_queries(sid, cams[views])
        try:
            ctx.score(sid, opts, out=s)
            objective = ctx.stats()["objective_sum"]
        except CsgsError as e:
            if e.status != CSGS_E_EMPTY:
                raise
            s.zero_()  # every query of this shard has A = 0: it contributes nothing
    else:
        s.zero_()
    ctx.sync()
    combine_shards(s, objective, opts.resolution if opts is not None else 0, dist,
                   lambda t, f: ctx.scale_scores(t, f), group)
    S = ctx.total_sensitivity(s)
    if not S > 0.0:
        raise CsgsError(CSGS_E_EMPTY, "every query has A = 0: total sensitivity is zero")
    return s, S
