"""Iterative pruning (Section IV-C) on the device, driven from the removal-effect pass.

Each iteration recomputes dMSE_k and I_k of the remaining splats over every view (the removal
effect), then ``potr_prune_select`` removes a budget's worth of the splats below dMSE_MAX, in
ascending order of the mapping function m, and ``potr_prune_apply`` takes them out of the scene
(opacity 0).  The budget spreads the candidates' importance over the remaining iterations, so
the last iteration removes every splat still below dMSE_MAX.
"""
from __future__ import annotations

import torch

from . import _binding as B

A_DEFAULT = 10.0
ITERATIONS_DEFAULT = 48


def dmse_max(q: float) -> float:
    """dMSE_MAX = 10^(-8.8 - 2q) (hyper-parameter table of the paper)."""
    return 10.0 ** (-8.8 - 2.0 * q)


class PruneController:
    """Alive mask and workspace of one pruning run over n splats."""

    def __init__(self, n: int, device="cuda", iterations: int = ITERATIONS_DEFAULT, q: float = 0.5,
                 a: float = A_DEFAULT, dmse_max_value: float | None = None):
        self.n = int(n)
        self.device = torch.device(device)
        self.iterations = int(iterations)
        self.a = float(a)
        self.dmse_max = float(dmse_max_value if dmse_max_value is not None else dmse_max(q))
        self.alive = torch.ones(self.n, dtype=torch.uint8, device=self.device)
        self.removed = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.ws = torch.empty(B.potr_prune_workspace_size(self.n), dtype=torch.uint8, device=self.device)
        self.it = 0

    @property
    def remaining(self) -> int:
        return self.iterations - self.it

    def select(self, dmse: torch.Tensor, importance: torch.Tensor, stream=None):
        """One controller iteration on the current dMSE / importance (device, float64 [n])."""
        if self.remaining < 1:
            raise RuntimeError("every pruning iteration has run")
        B.potr_prune_select(self.n, dmse, importance, self.alive, self.dmse_max, self.a, self.remaining,
                            self.removed, self.ws, stream)
        self.it += 1

    def apply(self, opacity_logits: torch.Tensor, stream=None):
        """Opacity 0 for every removed splat (its logit becomes -inf)."""
        B.potr_prune_apply(self.n, self.alive, opacity_logits, stream)

    def alive_count(self) -> int:
        return int(self.alive.sum().item())


def prune(batched, targets: torch.Tensor, controller: PruneController, iterations: int | None = None,
          on_iteration=None):
    """Run ``iterations`` controller iterations (default: all that remain) over a
    ``BatchedRemovalEffect`` whose scene tensors the controller edits in place.
    ``on_iteration(it, dmse, importance, controller)`` is called after each selection."""
    n = controller.n
    dev = controller.device
    dmse = torch.zeros(n, dtype=torch.float64, device=dev)
    imp = torch.zeros(n, dtype=torch.float64, device=dev)
    logits = batched.frames[0].scene["opacity_logits"]
    todo = controller.remaining if iterations is None else int(iterations)
    for _ in range(todo):
        dmse.zero_()
        imp.zero_()
        batched.step(targets, dmse, imp)
        controller.select(dmse, imp)
        controller.apply(logits)
        if on_iteration is not None:
            on_iteration(controller.it, dmse, imp, controller)
    return controller
