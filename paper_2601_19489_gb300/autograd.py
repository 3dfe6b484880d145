"""torch.autograd.Function around the forward blend and its backward kernel.

Forward: gs_preprocess -> gs_bin_sort -> gs_render_fwd; backward:
gs_render_bwd (per-Gaussian blend backward + preprocess backward).  The
workspace of `plan` carries the forward's state (sorted lists, checkpoints)
to the backward, so a plan serves one forward/backward pair at a time.
"""
from __future__ import annotations

import torch

from .api import Gaussians, Plan, gs_bin_sort, gs_preprocess, gs_render_bwd, gs_render_fwd


class GsRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, plan: Plan, cams, bg, sh_degree: int,
                load_balanced: bool = True):
        params = Gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(),
                           opacity_logits.contiguous(), sh.contiguous(), int(sh_degree))
        P = plan.pixels
        rgb = torch.empty(3 * P, device=means.device)
        disp = torch.empty(P, device=means.device)
        T = torch.empty(P, device=means.device)
        gs_preprocess(plan, params, cams)
        gs_bin_sort(plan, load_balanced)
        gs_render_fwd(plan, bg, rgb, disp, T)
        ctx.plan, ctx.cams, ctx.bg, ctx.sh_degree = plan, cams, bg, int(sh_degree)
        ctx.save_for_backward(*params.tensors(), rgb, disp)
        ctx.mark_non_differentiable(T)
        return rgb, disp, T

    @staticmethod
    def backward(ctx, g_rgb, g_disp, g_T):
        means, log_scales, quats, opacity_logits, sh, rgb, disp = ctx.saved_tensors
        params = Gaussians(means, log_scales, quats, opacity_logits, sh, ctx.sh_degree)
        grads = params.zeros_like()
        if g_rgb is None:
            g_rgb = torch.zeros_like(rgb)
        gs_render_bwd(ctx.plan, params, ctx.cams, ctx.bg, rgb, disp, g_rgb.contiguous(),
                      g_disp.contiguous() if g_disp is not None else None, grads)
        return (*grads.tensors(), None, None, None, None, None)


def render(params: Gaussians, plan: Plan, cams, bg=(0.0, 0.0, 0.0), load_balanced: bool = True):
    """Differentiable render of all views of `plan`: flat planar colour (3P),
    blended disparity (P) and final transmittance (P)."""
    return GsRender.apply(params.means, params.log_scales, params.quats, params.opacity_logits, params.sh,
                          plan, cams, bg, params.sh_degree, load_balanced)
