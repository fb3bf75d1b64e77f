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
    """Adam fine-tuning of a scene (dict of device tensors, updated in place) on its views.

    Adam takes its step count from a device counter and its per-step factors from a table
    (potr_adam_step_scheduled), so with ``graphs`` each view's whole iteration -- preprocess,
    binning, render, loss gradient, backward, Adam -- is captured once in a CUDA graph (after one
    eager iteration of that view) and replayed; re-planning a view's capacity drops its graph.
    Both forms issue the same kernels and give the same bits."""

    def __init__(self, scene: dict, cams_rec: np.ndarray, targets: list, lam: float = 0.2, extent: float = 1.0,
                 lr=None, device="cuda", check_every: int = 25, graphs: bool = True, **cfg):
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
        self.step_counter = torch.zeros(1, dtype=torch.int32, device=self.device)  # Adam steps done
        self.sched, self.sched_rows = None, 0
        self.use_graphs = bool(graphs)
        self._graphs = [None] * len(self.frames)
        self._warm = [False] * len(self.frames)

    def _buffers(self, fr):
        key = fr.total_pixels
        if key not in self._bufs:
            self._bufs[key] = (fr.image_buffer(), fr.pixel_buffer(), fr.pixel_buffer(torch.int32), fr.image_buffer())
        return self._bufs[key]

    def _ensure_schedule(self, steps: int):
        """A device table of Adam's per-step factors covering ``steps`` steps (regrowing it drops
        the captured graphs, which hold its address)."""
        if steps <= self.sched_rows:
            return
        rows = max(steps, 2 * self.sched_rows, 1024)
        table = B.potr_adam_schedule(1, rows, self.lr)
        self.sched = torch.from_numpy(table.reshape(-1)).to(self.device)
        self.sched_rows = rows
        self._graphs = [None] * len(self.frames)

    def _iteration(self, view: int):
        """The device work of one iteration on the current stream (no host synchronisation)."""
        fr = self.frames[view]
        img, tf, nl, dL = self._buffers(fr)
        fr.preprocess()
        fr.bin_sort()
        fr.render(img, tf, nl)
        self.loss.zero_()
        fr.loss_grad(img, self.targets[view], self.lam, dL, self.loss)
        fr.render_backward(dL, self.grads, tf, nl)
        B.potr_adam_step_scheduled(self.scene, self.grads, self.m, self.v, self.n, self.sched, self.sched_rows,
                                   self.step_counter)

    def step(self, view: int):
        """One iteration on one view: forward, loss gradient, backward, Adam."""
        self.t += 1
        self._ensure_schedule(self.t)
        if self.check_every and self.t % self.check_every == 0:
            self.ensure_capacity()
        g = self._graphs[view]
        if g is not None:
            g.replay()
            return
        self._iteration(view)
        if self.use_graphs and self._warm[view]:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):  # records only; the next iteration of this view replays it
                self._iteration(view)
            self._graphs[view] = g
        self._warm[view] = True

    def ensure_capacity(self):
        """Re-plan every frame whose instances outgrew its capacity (the parameters move)."""
        for v, f in enumerate(self.frames):
            code, _ = f.status.tolist()
            if code == B.POTR_ERR_CAPACITY:
                f.plan(1.2)
                self._graphs[v] = None
                self._warm[v] = False

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
