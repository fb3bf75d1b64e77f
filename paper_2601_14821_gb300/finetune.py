"""Fine-tuning loop of POTR-FT (Section IV-F) on the device.

The paper fine-tunes with "the original 3DGS training routine": per iteration one training view
is rendered, the photometric loss against its image is differentiated (here L = (1 - lambda)
mean|c - c_t| + lambda mean (c - c_t)^2, lambda = 0.2), the gradient flows back through the
rasterizer and the projection (potr_render_backward), and Adam updates every parameter group
with its own learning rate (potr_adam_step).  The learning rates are the 3DGS routine's: means
1.6e-4 x scene extent, log-scales 5e-3, quaternions 1e-3, opacity logits 5e-2, SH DC 2.5e-3,
SH rest 2.5e-3 / 20, held constant over the short fine-tuning run.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B
from .pipeline import RemovalEffectFrame

LR_3DGS = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-3 / 20.0)  # means, log_scales, quats, opacity, SH DC, SH rest


class FineTuner:
    """Adam fine-tuning of a scene (dict of device tensors, updated in place) on its views."""

    def __init__(self, scene: dict, cams_rec: np.ndarray, targets: list, lam: float = 0.2, extent: float = 1.0,
                 lr=None, device="cuda", check_every: int = 25, **cfg):
        self.scene = scene
        self.device = torch.device(device)
        cams_rec = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)
        self.frames = [RemovalEffectFrame(scene, cams_rec[v:v + 1], device=self.device, with_importance=False, **cfg)
                       for v in range(cams_rec.shape[0])]
        for f in self.frames:
            f.plan(1.2)
        self.targets = targets
        self.lam = float(lam)
        lr = list(lr if lr is not None else LR_3DGS)
        lr[0] *= float(extent)
        self.lr = lr
        self.n = self.frames[0].n
        self.m = {k: torch.zeros_like(t) for k, t in scene.items()}
        self.v = {k: torch.zeros_like(t) for k, t in scene.items()}
        self.grads = {k: torch.empty_like(t) for k, t in scene.items()}
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.t = 0
        self.check_every = int(check_every)
        self._bufs = {}

    def _buffers(self, fr):
        key = fr.total_pixels
        if key not in self._bufs:
            self._bufs[key] = (fr.image_buffer(), fr.pixel_buffer(), fr.pixel_buffer(torch.int32), fr.image_buffer())
        return self._bufs[key]

    def step(self, view: int, stream=None):
        """One iteration on one view: forward, loss gradient, backward, Adam."""
        fr = self.frames[view]
        img, tf, nl, dL = self._buffers(fr)
        fr.preprocess(stream)
        fr.bin_sort(stream)
        self.t += 1
        if self.check_every and self.t % self.check_every == 0:
            self.ensure_capacity()
        fr.render(img, tf, nl, stream)
        self.loss.zero_()
        fr.loss_grad(img, self.targets[view], self.lam, dL, self.loss, stream)
        fr.render_backward(dL, self.grads, tf, nl, stream)
        B.potr_adam_step(self.scene, self.grads, self.m, self.v, self.n, self.t, self.lr, stream=stream)

    def ensure_capacity(self):
        """Re-plan every frame whose instances outgrew its capacity (the parameters move)."""
        for f in self.frames:
            code, _ = f.status.tolist()
            if code == B.POTR_ERR_CAPACITY:
                f.plan(1.2)

    def run(self, iterations: int, order=None, seed: int = 0):
        """``iterations`` steps over the views (a seeded random view per step, as 3DGS draws
        them, unless ``order`` is given); returns the loss of the last step."""
        rng = np.random.default_rng(seed)
        views = order if order is not None else rng.integers(0, len(self.frames), size=iterations)
        for it in range(iterations):
            self.step(int(views[it % len(views)]))
        return float(self.loss.item())


def potr_ft(scene: dict, cams_rec: np.ndarray, targets: list, eyes, q: float = 0.5, cycles: int = 2,
            iterations: int = 500, lam: float = 0.2, extent: float = 1.0, seed: int = 0, compress: bool = True,
            **cfg) -> dict:
    """POTR-FT (Section IV-F): ``cycles`` rounds of decode -> fine-tune -> encode, every step on the
    device (the codec's zlib stage is lossless and is applied once, to the final bitstream, on the
    host; ``compress=False`` leaves it to the caller).  The scene must hold only live splats
    (compact a pruned scene first).  Returns the final bitstream (raw, and compressed unless
    ``compress`` is False), the fine-tuned scene before its last encoding, and the loss after
    each cycle's fine-tuning."""
    from .codec import Encoder, encode, params, roundtrip

    p = params(q)
    losses = []
    for c in range(cycles):
        decoded, _ = roundtrip(scene, eyes, p=p)
        ft = FineTuner(decoded, cams_rec, targets, lam=lam, extent=extent, device=scene["means"].device, **cfg)
        losses.append(ft.run(iterations, seed=seed + c))
        scene = ft.scene
    if compress:
        out = encode(scene, eyes, p=p)
    else:
        enc = Encoder(int(scene["means"].shape[-1]), scene["means"].device)
        enc.run(scene, eyes, p)
        out = {"raw": enc.stream(p), "order": enc.order.cpu().numpy()}
    out["scene"] = scene
    out["losses"] = losses
    return out
