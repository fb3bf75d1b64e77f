"""Pins of the pruning-controller oracle (Section IV-C) against facts fixed outside it."""
import math

import numpy as np
import pytest

from oracle import prune


def test_mapping_function_closed_forms():
    a = prune.A_DEFAULT
    assert prune.m_map(0.0) == 0.0 and math.copysign(1.0, prune.m_map(-0.0)) == 1.0
    for x in (1e-9, 0.3, 1.0, 7.5):
        assert prune.m_map(x) == x
    # x < 0: m(x) = y  <=>  x = -(a y^2 + 2 y) / 2 (square both sides of sqrt(1 - 2ax) = a y + 1)
    for y in (1e-6, 0.01, 0.5, 1.0, 3.0):
        x = -(a * y * y + 2.0 * y) / 2.0
        assert prune.m_map(x) == pytest.approx(y, rel=1e-12)
    # V-shaped at 0 with slope -1 on the left; negative effects cost less than positive ones
    eps = 1e-8
    assert prune.m_map(-eps) == pytest.approx(eps, rel=1e-6)
    for x in (0.1, 1.0, 5.0):
        assert prune.m_map(-x) < prune.m_map(x)
    assert prune.dmse_max(0.5) == pytest.approx(10 ** -9.8, rel=1e-14)


def test_hand_worked_iteration():
    # dMSE_MAX = 1, a = 10.  Candidates: every splat but 2 (dMSE 2.0 >= 1).  m values: splat 5
    # 0, splat 3 0.1, splat 1 (sqrt(7)-1)/10 = 0.1646, splat 0 0.5, splat 4 (sqrt(101)-1)/10 =
    # 0.905.  Sum of I over candidates 0.75.
    dmse = [0.5, -0.3, 2.0, 0.1, -5.0, 0.0]
    imp = [0.1, 0.2, 0.3, 0.05, 0.25, 0.15]
    alive = [True] * 6
    # two iterations left: B = 0.375; cumulative I in m order 0.15, 0.20, 0.40 -> S = {5, 3, 1}
    removed, budget, total, order = prune.select(dmse, imp, alive, 1.0, 2)
    assert order == [5, 3, 1]
    assert budget == (prune.quantize_importance(np.array(imp))[[0, 1, 3, 4, 5]].sum()) // 2
    assert np.array_equal(np.nonzero(removed)[0], [1, 3, 5])
    # last iteration: every candidate goes, in m order
    removed, budget, total, order = prune.select(dmse, imp, alive, 1.0, 1)
    assert order == [5, 3, 1, 0, 4] and not removed[2]
    # a splat already removed is no candidate
    removed, *_ = prune.select(dmse, imp, [True, False, True, True, True, True], 1.0, 2)
    assert not removed[1]


def test_threshold_is_strict_and_bad_importances_count_zero():
    """Candidates have dMSE_k strictly below dMSE_MAX (a splat exactly at it stays); an importance
    that is negative or NaN adds nothing to the budget."""
    removed, budget, total, order = prune.select([1.0, 0.5, 0.999999], [0.3, 0.2, 0.1], [True] * 3, 1.0, 1)
    assert order == [1, 2] and not removed[0]
    q = prune.quantize_importance(np.array([-1e-3, np.nan, 0.25, 0.0, -0.0]))
    assert q.tolist() == [0, 0, 2 ** 38, 0, 0]
    removed, budget, *_ = prune.select([0.1, 0.2], [-0.5, 0.25], [True, True], 1.0, 1)
    assert budget == 2 ** 38 and removed.tolist() == [True, True]


def _numpy_select(dmse, imp, alive, dmax, remaining, a=prune.A_DEFAULT):
    """The same rule through numpy: lexsort on (m, index), cumulative sum, searchsorted."""
    q = np.floor(np.asarray(imp) * 2.0 ** 40).astype(np.int64)
    cand = np.nonzero(np.asarray(alive) & (np.asarray(dmse) < dmax))[0]
    x = np.asarray(dmse)[cand] / dmax
    with np.errstate(invalid="ignore"):
        m = np.where(x >= 0, x + 0.0, (np.sqrt(1.0 - (2.0 * a) * x) - 1.0) / a)
    order = cand[np.lexsort((cand, m))]
    budget = int(q[cand].sum()) // remaining
    if budget <= 0:
        return np.zeros(len(dmse), bool)
    c = np.cumsum(q[order])
    stop = int(np.searchsorted(c, budget, side="left")) + 1  # first prefix whose sum >= B
    out = np.zeros(len(dmse), bool)
    out[order[:stop]] = True
    return out


def test_against_numpy_formulation_and_invariants():
    rng = np.random.default_rng(8)
    for trial in range(300):
        n = int(rng.integers(1, 60))
        dmax = 10.0 ** rng.uniform(-11, -8)
        dmse = rng.normal(0, 1, n) * dmax * rng.choice([0.1, 1.0, 10.0])
        dmse[rng.random(n) < 0.1] = 0.0
        dmse[rng.random(n) < 0.05] = -0.0
        imp = rng.exponential(1e-4, n) * (rng.random(n) < 0.9)
        if trial % 7 == 0:  # exact ties in m and in importance
            dmse[: n // 2] = dmse[0]
            imp[: n // 3] = imp[0]
        alive = rng.random(n) < 0.85
        R = int(rng.integers(1, 49))
        removed, budget, total, order = prune.select(dmse, imp, alive, dmax, R)
        assert np.array_equal(removed, _numpy_select(dmse, imp, alive, dmax, R))
        cand = alive & (dmse < dmax)
        assert not np.any(removed & ~cand)
        q = prune.quantize_importance(imp)
        if budget > 0 and removed.any():
            assert total >= budget or removed.sum() == cand.sum()
            assert total - q[order[-1]] < budget
        if R == 1 and budget > 0:
            # the last iteration removes every candidate up to the last one carrying importance
            # (trailing zero-importance candidates cannot change a reached budget)
            cidx = np.nonzero(cand)[0]
            x = dmse[cidx] / dmax
            ordr = [k for _, k in sorted((prune.m_map(v), int(k)) for v, k in zip(x, cidx))]
            last = max(i for i, k in enumerate(ordr) if q[k] > 0)
            assert removed[ordr[: last + 1]].all() and not removed[ordr[last + 1:]].any()


def test_loop_removes_every_candidate_once_effects_stay_put():
    # with effects that do not change between iterations, 48 iterations remove exactly the
    # splats below dMSE_MAX, a budget's worth (about 1/remaining of the candidates' importance)
    # per iteration
    rng = np.random.default_rng(4)
    n = 500
    dmax = 1e-9
    dmse = rng.normal(0, 2e-9, n)
    imp = rng.exponential(1e-3, n)
    hist = prune.run(lambda alive: (dmse, imp), n, 48, dmax)
    assert np.array_equal(~hist[-1], dmse < dmax)
    removed_per_it = [int((~hist[0]).sum())] + [int((hist[i - 1] & ~hist[i]).sum()) for i in range(1, 48)]
    assert all(r >= 0 for r in removed_per_it) and sum(removed_per_it) == int((dmse < dmax).sum())
