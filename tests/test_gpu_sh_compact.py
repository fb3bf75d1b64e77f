"""SH energy compaction on the device (potr_sh_compact) and the per-view importance it is
weighted by (potr_removal_effect's d_imp_view), against the oracles."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_close_abs_rel, build_frame, oracle_cfg, pack_targets
from oracle import sh_compact as oshc

pytestmark = pytest.mark.gpu

CFG = dict(tile_w=16, tile_h=16, batch=256)


@pytest.fixture(scope="module")
def run():
    import torch

    sc = synth.uniform_cube_scene(3000, 17)
    cams = synth.ring_cameras(12, 3.0, 0.3, (96, 96))
    fr = build_frame(sc, cams, **CFG)
    n, V = sc.n, len(cams)
    imp_view = torch.zeros(V * n, dtype=torch.float64, device="cuda")
    dmse = torch.zeros(n, dtype=torch.float64, device="cuda")
    tg = [np.zeros((3, c.height, c.width), np.float32) for c in cams]
    fr.removal_effect(pack_targets(fr, tg), dmse, None, imp_view=imp_view)
    torch.cuda.synchronize()
    return sc, cams, fr, imp_view, imp_view.cpu().numpy().reshape(V, n)


def test_per_view_importance_matches_oracle(run):
    sc, cams, fr, _, iv = run
    ocfg = oracle_cfg(CFG)
    act = oracle.activate(sc)
    for v in (0, 5, 11):
        pv = oracle.prepare_view(sc, cams[v], ocfg, act)
        _, imp = oracle.removal_effect(pv, pv["vals"], pv["ranges"], cams[v], ocfg, np.zeros((3, 96, 96), np.float32))
        assert_close_abs_rel(iv[v], imp / cams[v].pixels, 1e-4, 1e-9, f"I_k({v})")
        assert np.count_nonzero(imp) > 500


def _margins(kept, first, G, alpha, sf):
    """Distance of the oracle's integer decisions from their thresholds (cosines and roundings)."""
    if kept is None:
        return math.inf
    m = math.inf
    seen = [0]
    for i in range(1, 16):
        if G[i, i] <= 0:
            continue
        for j in seen:
            m = min(m, abs(abs(G[i, j]) / math.sqrt(G[i, i] * G[j, j]) - alpha))
        if i in kept:
            seen.append(i)
    for ch in range(3):
        for i in kept[1:]:
            t = 0.5 + first[i, ch] * sf
            m = min(m, abs(t - round(t)) if abs(t - round(t)) < 0.5 else 1.0)
    return m


@pytest.mark.parametrize("case", ["paper q=0.5", "weak regularisation"])
def test_compaction_matches_oracle(run, case):
    from paper_2601_14821_gb300.sh_compact import compact, params

    sc, cams, fr, imp_view, iv = run
    p = params(0.5) if case.startswith("paper") else {"lam": 1e-4, "alpha": 0.9, "sf": 51.0}
    rgb, ycocg, kept = compact(fr, imp_view, p=p)
    rgb, ycocg, kept = rgb.cpu().numpy(), ycocg.cpu().numpy(), kept.cpu().numpy().view(np.uint32)
    centres = np.array([oshc.camera_centre(c) for c in cams])
    seen = np.nonzero((iv > 0).sum(axis=0) >= 6)[0]
    pick = np.unique(np.concatenate([seen[:400], np.nonzero((iv > 0).sum(axis=0) == 0)[0][:20],
                                     np.nonzero((iv > 0).sum(axis=0) == 1)[0][:20]]))
    compared = skipped = 0
    for k in pick:
        Lp, kp, per_ch, first, G = oshc.compact_splat(sc.sh[:, :, k], sc.means[:, k], centres, iv[:, k], p["lam"],
                                                       p["alpha"], p["sf"])
        want_masks = [0, 0, 0, 0] if kp is None else [sum(1 << i for i in s) for s in [kp] + per_ch]
        if list(kept[:, k]) != want_masks:
            assert _margins(kp, first, G, p["alpha"], p["sf"]) < 1e-9, k  # only at a tie
            skipped += 1
            continue
        scale = max(1.0, np.abs(Lp).max())
        np.testing.assert_allclose(ycocg[:, :, k], Lp, rtol=0, atol=1e-9 * scale, err_msg=str(k))
        np.testing.assert_allclose(rgb[:, :, k], Lp @ oshc.YCOCG_TO_RGB.T, rtol=0, atol=2e-6 * scale)
        compared += 1
    assert compared >= 0.95 * len(pick) and skipped <= 2
    # the AC paths were exercised: some splats keep more than the DC in pass 2
    multi = sum(bin(int(x)).count("1") > 1 for x in kept[1][pick])
    if case.startswith("weak"):
        assert multi > 100
