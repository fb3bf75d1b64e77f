"""Spherical-harmonics energy compaction (Section IV-D) on the device.

``compact(frame, imp_view, q)`` takes the per-view importances I_k(s) of a frame's views (from
``RemovalEffectFrame.removal_effect(..., imp_view=...)``) and returns the compacted lighting
coefficients of every splat: in RGB (float32, the scene's SH layout, ready to render), in YCoCg
(float64, what the codec would quantise) and the kept-column masks.
"""
from __future__ import annotations

import math

import torch

from . import _binding as B


def params(q: float) -> dict:
    """lambda = 10^-q, alpha = sigmoid(3q), SF_SH = 1 + 100 q (hyper-parameter table)."""
    return {"lam": 10.0 ** (-q), "alpha": 1.0 / (1.0 + math.exp(-3.0 * q)), "sf": 1.0 + 100.0 * q}


def compact(frame, imp_view: torch.Tensor, q: float = 0.5, p: dict | None = None, stream=None):
    p = p or params(q)
    n = frame.n
    dev = frame.device
    sh_rgb = torch.empty(16 * 3 * n, dtype=torch.float32, device=dev)
    sh_ycocg = torch.empty(16 * 3 * n, dtype=torch.float64, device=dev)
    kept = torch.empty(4 * n, dtype=torch.int32, device=dev)
    B.potr_sh_compact(frame.scene_c, frame.frame, imp_view, p["lam"], p["alpha"], p["sf"], sh_rgb, sh_ycocg, kept,
                      stream)
    return sh_rgb.view(16, 3, n), sh_ycocg.view(16, 3, n), kept.view(4, n)
