"""torch.autograd wrapper of the rasterizer with a hand-written backward.

``render(ctx, g, cam, pose, xi)`` returns (rgb [3,H,W], depth [H,W],
alpha [H,W]) as differentiable tensors.  Gradients flow to every Gaussian
parameter and to ``xi``, the 6-vector (rho, phi) of a left perturbation
exp(xi^) T_wc of the world-to-camera pose (use ``xi = zeros(6,
requires_grad=True)`` to obtain the pose gradient of Sec. 3.5's tracking).

The forward saves only the per-pixel final transmittance and last
contributor index; the backward (gsr_render_backward) replays the tile
lists the context kept, or rebuilds them when another forward ran since or
when the context is in memory-saving mode.
"""
from __future__ import annotations

import torch

from . import api


class GaussianRender(torch.autograd.Function):
    @staticmethod
    def forward(fctx, rctx, cam, pose_q, pose_t, xi, mean, log_scale, quat, opacity_logit, rgb):
        g = api.GaussianParams(mean.detach().contiguous(), log_scale.detach().contiguous(),
                               quat.detach().contiguous(), opacity_logit.detach().contiguous(),
                               rgb.detach().contiguous())
        xi_h = xi.detach().double().cpu().numpy()
        q, t = api.pose_exp_left(pose_q, pose_t, xi_h) if abs(xi_h).max() > 0 else (pose_q, pose_t)
        pose = api.make_pose(q, t)
        out = api.render_forward(rctx, g, cam, pose)
        fctx.rctx, fctx.cam, fctx.pose, fctx.g = rctx, cam, pose, g
        fctx.saved = dict(final_T=out["final_T"], last_idx=out["last_idx"])
        fctx.mark_non_differentiable(out["final_T"])
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(fctx, d_rgb, d_depth, d_alpha):
        cont = lambda t: None if t is None else t.contiguous()
        grads, pose6 = api.render_backward(fctx.rctx, fctx.g, fctx.cam, fctx.pose, fctx.saved, cont(d_rgb),
                                           cont(d_depth), cont(d_alpha), want_params=True,
                                           want_pose=fctx.needs_input_grad[4])
        return (None, None, None, None, pose6, grads.mean, grads.log_scale, grads.quat, grads.opacity_logit,
                grads.rgb)


def render(rctx: api.Context, g: api.GaussianParams, cam, pose_q, pose_t, xi=None):
    """Differentiable render; returns (rgb, depth, alpha)."""
    if xi is None:
        xi = torch.zeros(6, device=g.mean.device)
    return GaussianRender.apply(rctx, cam, pose_q, pose_t, xi, g.mean, g.log_scale, g.quat, g.opacity_logit,
                                g.rgb)
