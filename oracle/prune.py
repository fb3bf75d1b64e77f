"""Pruning controller of POTR (Section IV-C, "Iterative pruning") -- plain reference.

TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and the benchmark's CPU
baseline; the CUDA library never calls it and shares no code with it.

One controller iteration, as Section IV-C defines it:
  * the controller aims to remove every splat with dMSE_k < dMSE_MAX (the candidates);
  * budget B = (1 / #remaining iterations) * sum of I_k over the candidates (pruning budget
    equation);
  * splats are added to the removal set S in ascending order of m(dMSE_k / dMSE_MAX), with
    m(x) = x for x >= 0 and (sqrt(1 - 2 a x) - 1) / a for x < 0 (mapping-function equation),
    until the budget is reached, i.e. until B <= sum over S of I_k (budget equation).

Readings (the paper is silent on them):
  * only candidates are added to S, so the last iteration removes exactly the candidates;
  * ties in m are broken by splat index (ascending);
  * importance is accounted in fixed point: q_k = floor(I_k * 2^40) as an integer, B =
    floor(sum q_k / R) with R the number of remaining iterations, and S grows while its q-sum
    is below B (B <= 0 gives an empty S).  Integer sums make the "budget reached" decision exact
    whatever order the sums are taken in, so it is the same on every implementation;
  * m is evaluated in binary64 with IEEE operations in the written order, and -0 maps to +0;
  * a = 10 (the value of the paper's mapping-function figure); dMSE_MAX = 10^(-8.8 - 2q) and 48
    iterations (hyper-parameter table).
"""
from __future__ import annotations

import math

import numpy as np

Q_BITS = 40
A_DEFAULT = 10.0
ITERATIONS_DEFAULT = 48


def dmse_max(q: float) -> float:
    """dMSE_MAX as a function of the quality parameter q (hyper-parameter table)."""
    return 10.0 ** (-8.8 - 2.0 * q)


def m_map(x: float, a: float = A_DEFAULT) -> float:
    """The mapping function m(x) of Section IV-C (binary64, operations in the written order)."""
    if x >= 0.0:
        return x + 0.0  # -0 -> +0
    return (math.sqrt(1.0 - (2.0 * a) * x) - 1.0) / a


def quantize_importance(imp) -> np.ndarray:
    """q_k = floor(I_k * 2^40) (the scaling by a power of two is exact); an importance that is
    not >= 0 (NaN) counts as 0."""
    imp = np.asarray(imp, np.float64)
    imp = np.where(imp >= 0.0, imp, 0.0)
    return np.floor(imp * float(1 << Q_BITS)).astype(np.int64)


def select(dmse, imp, alive, dmse_max_value: float, remaining: int, a: float = A_DEFAULT):
    """One controller iteration: returns (removed mask, budget B, q-sum of S, order of S)."""
    dmse = np.asarray(dmse, np.float64)
    alive = np.asarray(alive, bool)
    q = quantize_importance(imp)
    n = dmse.size
    cand = [k for k in range(n) if alive[k] and dmse[k] < dmse_max_value]
    budget = int(sum(int(q[k]) for k in cand)) // int(remaining)
    keyed = sorted(cand, key=lambda k: (m_map(dmse[k] / dmse_max_value, a), k))
    removed = np.zeros(n, bool)
    total = 0
    order = []
    for k in keyed:
        if budget <= total:  # budget reached
            break
        removed[k] = True
        order.append(k)
        total += int(q[k])
    return removed, budget, total, order


def run(step, n: int, iterations: int, dmse_max_value: float, a: float = A_DEFAULT):
    """The iterative loop: ``step(alive) -> (dmse, importance)`` recomputes the removal
    effects of the remaining splats; each iteration removes its S.  Returns the alive mask
    after every iteration."""
    alive = np.ones(n, bool)
    history = []
    for it in range(iterations):
        d, i = step(alive)
        removed, *_ = select(d, i, alive, dmse_max_value, iterations - it, a)
        alive = alive & ~removed
        history.append(alive.copy())
    return history
