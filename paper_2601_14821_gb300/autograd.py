"""torch.autograd bridge: the differentiable render of a frame for fine-tuning.

``RasterizeFn.apply(frame, store_transmittance, means, log_scales, quats, opacity_logits, sh)``
returns the frame's packed images (every view, planar [3][H][W] one after another) from
potr_preprocess + potr_bin_sort + potr_render, and its backward runs potr_render_backward.
With ``store_transmittance`` the forward keeps the final transmittance and n_last per pixel
for the backward; without it the backward recomputes them (no per-pixel storage).
"""
from __future__ import annotations

import torch

from . import _binding as B
from .pipeline import SCENE_KEYS, RemovalEffectFrame


class RasterizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, frame: RemovalEffectFrame, store_transmittance: bool, *params):
        scene = {k: p.detach().contiguous() for k, p in zip(SCENE_KEYS, params)}
        frame.bind_scene(scene)
        frame.preprocess()
        frame.bin_sort()
        if frame.status_code() == B.POTR_ERR_CAPACITY:
            frame.plan()
        img = frame.image_buffer()
        t_final = n_last = None
        if store_transmittance:
            t_final = frame.pixel_buffer()
            n_last = frame.pixel_buffer(torch.int32)
        frame.render(img, t_final, n_last)
        ctx.frame = frame
        ctx.scene = scene
        ctx.saved = (t_final, n_last)
        return img

    @staticmethod
    def backward(ctx, dL_dimg):
        frame = ctx.frame
        frame.bind_scene(ctx.scene)
        grads = {k: torch.empty_like(v) for k, v in ctx.scene.items()}
        t_final, n_last = ctx.saved
        frame.render_backward(dL_dimg.contiguous(), grads, t_final, n_last)
        return (None, None) + tuple(grads[k] for k in SCENE_KEYS)


def render(frame: RemovalEffectFrame, params: dict, store_transmittance: bool = True) -> torch.Tensor:
    return RasterizeFn.apply(frame, store_transmittance, *(params[k] for k in SCENE_KEYS))
