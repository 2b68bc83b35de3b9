"""torch.autograd.Function around the DDF network: forward = ddf_query (distance, logit),
backward = ddf_backward (weight gradient in the flat blob layout and d/d(o, w)), recomputing
activations on the device instead of keeping them from the forward."""

from __future__ import annotations

import torch

from .ddf import DDFNet


class DDFFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, net: DDFNet, weights: torch.Tensor, o: torch.Tensor, w: torch.Tensor):
        net.set_weights(weights.detach().contiguous())
        out = net.query(o.contiguous(), w.contiguous())
        ctx.net = net
        ctx.save_for_backward(weights, o, w)
        ctx.mark_non_differentiable(out["hit"])
        return out["dist"], out["logit"], out["hit"]

    @staticmethod
    def backward(ctx, gdist, glogit, _ghit):
        weights, o, w = ctx.saved_tensors
        net = ctx.net
        net.set_weights(weights.detach().contiguous())
        need_in = ctx.needs_input_grad[2] or ctx.needs_input_grad[3]
        gd = gdist.contiguous() if gdist is not None else torch.zeros(o.shape[0], device=o.device)
        gl = glogit.contiguous() if glogit is not None else torch.zeros(o.shape[0], device=o.device)
        gw, gin = net.backward(o.contiguous(), w.contiguous(), gd, gl, need_input=need_in)
        go = gin[:, :3] if need_in else None
        gwd = gin[:, 3:] if need_in else None
        return None, gw, go, gwd


def ddf_apply(net: DDFNet, weights: torch.Tensor, o: torch.Tensor, w: torch.Tensor):
    """(dist, logit, hit) of the network with differentiable `weights` (flat blob)."""
    return DDFFunction.apply(net, weights, o, w)
