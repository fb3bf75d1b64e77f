"""Adam step of the fine-tuning loop (Section IV-F: the original 3DGS training routine) -- plain
reference.  TEST INFRASTRUCTURE ONLY.

One step on parameter p with gradient g (Kingma & Ba, "Adam", 2015), in the form of PyTorch's
implementation that the 3DGS training routine uses (eps added to the bias-corrected root):
    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    p <- p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps).
Binary64.  Parameter groups of a scene (learning rates per group): means, log_scales, quats,
opacity_logits, SH DC (the first 3 of the 48 SH planes), SH rest.
"""
from __future__ import annotations

import numpy as np

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest")


def step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15):
    """In place on float64 arrays p, m, v (g read only); t >= 1 is the step number."""
    m *= b1
    m += (1.0 - b1) * g
    v *= b2
    v += (1.0 - b2) * g * g
    bc1 = 1.0 - b1 ** t
    bc2 = 1.0 - b2 ** t
    denom = np.sqrt(v) / np.sqrt(bc2) + eps
    p -= (lr / bc1) * m / denom


def split_groups(scene: dict) -> dict:
    """Views of the six parameter groups of a scene dict of SoA arrays (sh is [16][3][n])."""
    sh = scene["sh"].reshape(48, -1)
    return {"means": scene["means"], "log_scales": scene["log_scales"], "quats": scene["quats"],
            "opacity_logits": scene["opacity_logits"], "sh_dc": sh[:3], "sh_rest": sh[3:]}
