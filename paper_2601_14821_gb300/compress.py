"""The whole POTR compression of a trained scene on the device, as one call.

``compress(scene, cams_rec)`` chains the paper's stages in their order:

1. targets: the render of the unpruned scene (unless the caller gives them);
2. iterative pruning (Section IV-C): each iteration recomputes dMSE_k and I_k over every view and
   the controller removes a budget's worth of splats below dMSE_MAX;
3. SH energy compaction (Section IV-D) of the pruned scene from its per-view importances;
4. the live splats, with their compacted SH coefficients, are encoded (Section IV-E), or go
   through ``ft_cycles`` POTR-FT cycles of decode -> fine-tune -> encode (Section IV-F).

Every stage runs in ``libpotr.so``; the host only assembles the bitstream and applies zlib.
"""
from __future__ import annotations

import numpy as np
import torch

from .batched import BatchedRemovalEffect
from .codec import encode
from .finetune import potr_ft
from .pipeline import RemovalEffectFrame
from .prune import ITERATIONS_DEFAULT, PruneController, prune
from .sh_compact import compact
from .sh_compact import params as sh_params


def camera_centres(cams_rec: np.ndarray) -> np.ndarray:
    """Eye of every camera in a packed record array ({w2c[12], fx, fy, cx, cy, width, height}):
    with the world-to-camera map x_c = R x + t, the eye is the point mapped to 0, c = -R^T t."""
    rec = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)
    W = rec[:, :12].astype(np.float64).reshape(-1, 3, 4)
    return -np.einsum("vji,vj->vi", W[:, :, :3], W[:, :, 3])


def view_images(cams_rec: np.ndarray, images: torch.Tensor) -> list:
    """Split a packed image buffer (every view's 3 x height x width block, in view order) into
    per-view flat tensors."""
    rec = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)
    wh = rec[:, 16:18].copy().view(np.int32).astype(np.int64)
    out, off = [], 0
    for w, h in wh:
        out.append(images[off: off + 3 * w * h])
        off += 3 * w * h
    return out


def compress(scene: dict, cams_rec: np.ndarray, targets: torch.Tensor | None = None, q: float = 0.5,
             iterations: int = ITERATIONS_DEFAULT, ft_cycles: int = 0, ft_iterations: int = 500,
             views_per_chunk: int = 16, level: int = 6, lam: float = 0.2, extent: float = 1.0, seed: int = 0,
             dmse_max_value: float | None = None, eyes=None, **cfg) -> dict:
    """Prune, compact and encode ``scene`` (dict of float32 device planes, as ``scene_to_device``
    makes) seen from the cameras of ``cams_rec``.  The scene's opacity logits are edited in place
    (a removed splat's becomes -inf).  ``targets`` is a packed image buffer (3 * total pixels)
    and defaults to the unpruned render; ``dmse_max_value`` overrides the threshold
    10^(-8.8 - 2q); ``eyes`` ([V][3]) are the viewpoints the codec's position tolerance is taken
    from, by default the cameras' centres.  Returns the raw and zlib-compressed bitstream, the
    encoded scene (live splats only, in input order), the indices of the live splats, and the
    splat count after each pruning iteration."""
    rec = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)
    dev = scene["means"].device
    n = int(scene["means"].shape[-1])
    be = BatchedRemovalEffect(scene, rec, views_per_chunk=views_per_chunk, device=dev, **cfg)
    be.plan()
    if targets is None:
        targets = torch.empty(3 * be.total_pixels, dtype=torch.float32, device=dev)
        be.render(targets)
    ctrl = PruneController(n, device=dev, iterations=iterations, q=q, dmse_max_value=dmse_max_value)
    removed = []
    prune(be, targets, ctrl, on_iteration=lambda it, dmse, imp, c: removed.append(c.removed.clone()))
    counts = [int(x) for x in n - np.cumsum(torch.cat(removed).cpu().numpy())] if removed else []

    # per-view importances of the pruned scene over all views in one frame, then SH compaction
    if len(be.frames) == 1:
        frame = be.frames[0]
        frame.preprocess()
        frame.bin_sort()
    else:
        frame = RemovalEffectFrame(scene, rec, device=dev, **cfg)
        frame.plan()
    imp_view = torch.zeros(frame.n_views * n, dtype=torch.float64, device=dev)
    dmse = torch.zeros(n, dtype=torch.float64, device=dev)
    frame.removal_effect(targets, dmse, None, imp_view=imp_view)
    sh_rgb, _, _ = compact(frame, imp_view, p=sh_params(q))

    keep = torch.nonzero(ctrl.alive, as_tuple=False).flatten()
    sub = {k: t[..., keep].contiguous() for k, t in scene.items() if k != "sh"}
    sub["sh"] = sh_rgb[..., keep].contiguous()
    eyes = camera_centres(rec) if eyes is None else np.asarray(eyes, np.float64).reshape(-1, 3)
    if ft_cycles > 0:
        out = potr_ft(sub, rec, view_images(rec, targets), eyes, q=q, cycles=ft_cycles, iterations=ft_iterations,
                      lam=lam, extent=extent, seed=seed, **cfg)
    else:
        out = encode(sub, eyes, q=q, level=level)
        out["scene"] = sub
    out["keep"] = keep
    out["alive_after_iteration"] = counts
    return out
