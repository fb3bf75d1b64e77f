"""The pruning controller on the device (potr_prune_select / potr_prune_apply) against the
controller oracle (Section IV-C), on random effects and inside the iterative loop."""
import numpy as np
import pytest

import synth
from oracle import prune as oprune

pytestmark = pytest.mark.gpu


def _controller(n, **kw):
    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.prune import PruneController

    build.build()
    return PruneController(n, **kw)


@pytest.mark.parametrize("n", [1, 37, 5000, 300_000])
def test_select_matches_oracle_on_random_effects(n):
    import torch

    rng = np.random.default_rng(n)
    for trial in range(4):
        dmax = 10.0 ** rng.uniform(-11, -8)
        dmse = rng.normal(0, 1, n) * dmax * [0.1, 1.0, 3.0, 10.0][trial]
        dmse[rng.random(n) < 0.1] = 0.0
        dmse[rng.random(n) < 0.05] = -0.0
        dmse[rng.random(n) < 0.02] = np.nan
        if trial == 2:
            dmse[: n // 2] = dmse[0]  # a long run of equal m: ties by index
        imp = rng.exponential(1e-6, n) * (rng.random(n) < 0.9)
        imp[rng.random(n) < 0.01] = np.nan
        alive = rng.random(n) < 0.85
        R = [48, 7, 2, 1][trial]
        ctrl = _controller(n, iterations=R, dmse_max_value=dmax)
        ctrl.alive.copy_(torch.from_numpy(alive.astype(np.uint8)))
        d = torch.from_numpy(dmse).cuda()
        i = torch.from_numpy(imp).cuda()
        ctrl.select(d, i)
        torch.cuda.synchronize()
        want, budget, total, order = oprune.select(dmse, imp, alive, dmax, R)
        got = ctrl.alive.cpu().numpy().astype(bool)
        assert np.array_equal(got, alive & ~want), (n, trial)
        assert int(ctrl.removed.item()) == int(want.sum())


def test_pruning_loop_matches_oracle_iteration_by_iteration():
    """The tiny scene, six iterations: every selection equals the oracle's on the same device
    effects; pruned splats have zero effect and importance afterwards; the last iteration leaves
    no splat below dMSE_MAX."""
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.prune import PruneController, prune
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    w = synth.workload("tiny")
    scene = scene_to_device(w.scene)
    be = BatchedRemovalEffect(scene, synth.cameras_to_array(w.cameras), tile_w=16, tile_h=16, batch=256)
    be.plan()
    targets = torch.empty(3 * be.total_pixels, dtype=torch.float32, device="cuda")
    be.render(targets)  # the target is the render before pruning
    # dMSE_MAX at the median |dMSE| of the unpruned scene, so that many splats are candidates
    d0 = torch.zeros(w.scene.n, dtype=torch.float64, device="cuda")
    i0 = torch.zeros_like(d0)
    be.step(targets, d0, i0)
    dmax = float(np.median(np.abs(d0.cpu().numpy())))
    ctrl = PruneController(w.scene.n, iterations=6, dmse_max_value=dmax)
    seen = {"alive": np.ones(w.scene.n, bool)}

    def check(it, dmse, imp, c):
        d = dmse.cpu().numpy()
        i = imp.cpu().numpy()
        before = seen["alive"]
        assert np.all(d[~before] == 0.0) and np.all(i[~before] == 0.0), it
        want, *_ = oprune.select(d, i, before, dmax, 6 - (it - 1))
        after = c.alive.cpu().numpy().astype(bool)
        assert np.array_equal(after, before & ~want), it
        if it == 6:
            assert not np.any(after & (d < dmax))
        seen["alive"] = after

    prune(be, targets, ctrl, on_iteration=check)
    assert ctrl.it == 6 and 0 < ctrl.alive_count() < w.scene.n
