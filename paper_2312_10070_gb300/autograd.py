"""torch.autograd wrapper of the rasterizer with a hand-written backward.

``render(ctx, g, cam, pose, xi)`` returns (rgb [3,H,W], depth [H,W],
alpha [H,W]) as differentiable tensors.  Gradients flow to every Gaussian
parameter and to ``xi``, the 6-vector (rho, phi) of a left perturbation
exp(xi^) T_wc of the world-to-camera pose (use ``xi = zeros(6,
requires_grad=True)`` to obtain the pose gradient of Sec. 3.5's tracking).
``xi`` stays on the device: the perturbed pose is formed by
gsr_render_forward_xi and the backward returns dL/dxi through the SE(3) left
Jacobian (gsr_render_backward_xi), so neither pass synchronises with the host.

The forward saves only the per-pixel final transmittance and last
contributor index; the backward (gsr_render_backward_xi) replays the tile
lists the context kept, or rebuilds them when another forward ran since or
when the context is in memory-saving mode.
"""
from __future__ import annotations

import torch

from . import api


class GaussianRender(torch.autograd.Function):
    @staticmethod
    def forward(fctx, rctx, cam, pose, xi, mean, log_scale, quat, opacity_logit, rgb):
        g = api.GaussianParams(mean.detach().contiguous(), log_scale.detach().contiguous(),
                               quat.detach().contiguous(), opacity_logit.detach().contiguous(),
                               rgb.detach().contiguous())
        xi_d = xi.detach().to(torch.float32).contiguous()
        out = api.render_forward(rctx, g, cam, pose, xi=xi_d)
        fctx.rctx, fctx.cam, fctx.pose, fctx.g, fctx.xi = rctx, cam, pose, g, xi_d
        fctx.saved = dict(final_T=out["final_T"], last_idx=out["last_idx"])
        fctx.mark_non_differentiable(out["final_T"])
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(fctx, d_rgb, d_depth, d_alpha):
        cont = lambda t: None if t is None else t.contiguous()
        grads, d_xi = api.render_backward(fctx.rctx, fctx.g, fctx.cam, fctx.pose, fctx.saved, cont(d_rgb),
                                          cont(d_depth), cont(d_alpha), want_params=True,
                                          want_pose=fctx.needs_input_grad[3], xi=fctx.xi)
        return (None, None, None, d_xi, grads.mean, grads.log_scale, grads.quat, grads.opacity_logit, grads.rgb)


def render(rctx: api.Context, g: api.GaussianParams, cam, pose_q, pose_t, xi=None):
    """Differentiable render at exp(xi^) (q, t); returns (rgb, depth, alpha)."""
    if xi is None:
        xi = torch.zeros(6, device=g.mean.device)
    return GaussianRender.apply(rctx, cam, api.make_pose(pose_q, pose_t), xi, g.mean, g.log_scale, g.quat,
                                g.opacity_logit, g.rgb)
