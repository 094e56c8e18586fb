"""Short post-pruning recovery (the paper's "short recovery" finetune, Sec. 4): the
weighted coreset's means, SH colours and opacity logits are fitted to renders of the
full scene with the library's renderer and its hand-written backward.

`CoresetRender` is a torch.autograd.Function whose forward is csgs_render of the
weighted pruned scene and whose backward is csgs_render_backward; the Adam updates run
in the library's kernel (csgs_adam_update).  This module only sequences those calls.
"""
from __future__ import annotations

import numpy as np


def _autograd_function():
    import torch

    class CoresetRender(torch.autograd.Function):
        @staticmethod
        def forward(fctx, means, sh, logits, ctx, sid, view, log_scales, quats, idx, w, H, W, opts):
            ctx.update_scene(sid, means.detach(), log_scales, quats, logits.detach(), sh.detach())
            img = ctx.render(sid, view, idx=idx, w=w, H=H, W=W, opts=opts)
            fctx.save_for_backward(idx, w)
            fctx.args = (ctx, sid, view, opts, means.shape, sh.shape, logits.shape)
            return img

        @staticmethod
        def backward(fctx, grad_img):
            idx, w = fctx.saved_tensors
            ctx, sid, view, opts, ms, ss, ls = fctx.args
            gm = torch.zeros(ms, dtype=torch.float32, device=grad_img.device)
            gs = torch.zeros(ss, dtype=torch.float32, device=grad_img.device)
            gl = torch.zeros(ls, dtype=torch.float32, device=grad_img.device)
            ctx.render_backward(sid, view, grad_img.contiguous(), gm, gs, gl, idx=idx, w=w, opts=opts)
            return gm, gs, gl, None, None, None, None, None, None, None, None, None, None

    return CoresetRender


_CR = None


def coreset_render(ctx, sid, view, means, sh, logits, log_scales, quats, idx, w, H, W, opts=None):
    """Differentiable render of the weighted pruned scene (idx, w) w.r.t. means, SH and logits."""
    global _CR
    if _CR is None:
        _CR = _autograd_function()
    return _CR.apply(means, sh, logits, ctx, sid, view, log_scales, quats, idx, w, H, W, opts)


def finetune(ctx, sid, cams, params: dict, idx, w, targets, steps: int, lr_means=1e-3, lr_colour=1e-3,
             lr_opacity=5e-3, seed: int = 0, opts=None, log_every: int = 0, callback=None):
    """Adam on means, SH and opacity logits, one seeded-random view per step, loss = mean
    absolute error against the target render of that view.  params: device tensors
    means [3,N], log_scales [3,N], quats [4,N], opacity_logits [N], sh [K,3,N] of the
    scene `sid` (updated in place).  callback(step) runs after each step's update (the
    library's copy of the scene is refreshed only by the next step's forward, so a callback
    that renders calls ctx.update_scene first).  Returns the per-step losses."""
    import torch

    cams = np.asarray(cams, dtype=np.float32).reshape(-1, 20)
    rng = np.random.default_rng(seed)
    trainable = {"means": lr_means, "sh": lr_colour, "opacity_logits": lr_opacity}
    state = {k: (torch.zeros_like(params[k]), torch.zeros_like(params[k])) for k in trainable}
    losses = []
    for step in range(1, steps + 1):
        v = int(rng.integers(0, cams.shape[0]))
        H, W = int(cams[v][17]), int(cams[v][16])
        leaves = {k: params[k].detach().requires_grad_(True) for k in trainable}
        img = coreset_render(ctx, sid, v, leaves["means"], leaves["sh"], leaves["opacity_logits"],
                             params["log_scales"], params["quats"], idx, w, H, W, opts)
        loss = (img - targets[v]).abs().mean()
        loss.backward()
        for k, lr in trainable.items():
            m, vv = state[k]
            ctx.adam_update(params[k], leaves[k].grad.contiguous(), m, vv, lr, step)
        losses.append(float(loss.detach()))
        if log_every and step % log_every == 0:
            print(f"step {step} loss {losses[-1]:.5f}")
        if callback is not None:
            callback(step)
    ctx.update_scene(sid, params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                     params["sh"])
    return losses
