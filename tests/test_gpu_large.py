"""Parity on the largest workload's shapes: 1920x1080 views of the 6M-splat scene (shell radius
20) in the benchmark's 8-view chunks, and a single frame of 300 such views (2,448,000 global
tiles: 22 tile bits, three tile-partition passes).

The oracle cannot redo these frames; it checks what it can compute one view or one tile at a
time: a view's preprocess and complete binning/sort bit for bit (inside its frame: tile base and
value base of its position), and the image, transmittance, n_last and per-(tile, splat) removal
partials of sampled tiles of that view.  Targets: the oracle's render of the sampled view plus
N(0, 0.01) noise; a flat grey image for the others (their outputs are not compared)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (assert_close_abs_rel, assert_close_rel, assert_removal_close, frame_outputs, oracle_cfg, pack_targets,
                      view_slice)

pytestmark = pytest.mark.gpu

CFG = dict(tile_w=16, tile_h=16, batch=128)


def _targets(scene, cams, checked, seed):
    ocfg = oracle_cfg(CFG)
    out = []
    for v, c in enumerate(cams):
        if v in checked:
            pv = oracle.prepare_view(scene, c, ocfg)
            img, *_ = oracle.render(pv, pv["vals"], pv["ranges"], c, ocfg)
            out.append((img + synth.target_noise(img.shape, 0.01, seed, v)).astype(np.float32))
        else:
            out.append(np.full((3, c.height, c.width), 0.3, np.float32))
    return out


def _check_view(fr, res, scene, cam, v, tg, rng, n_tiles_sampled=20):
    """View v of frame fr: binning bit-exact, then sampled tiles' render and removal partials."""
    ocfg = oracle_cfg(CFG)
    n = scene.n
    act = oracle.activate(scene)
    pv = oracle.project(scene, act[0], cam, ocfg, act[1])
    pv["opacity"] = act[1]
    touched = fr.touched.cpu().numpy().view(np.uint32)
    assert np.array_equal(touched[v * n:(v + 1) * n], pv["touched"])
    m = fr.instance_count()
    tiles = fr.tiles[:m].cpu().numpy().view(np.uint32)
    vals = fr.vals[:m].cpu().numpy().view(np.uint32)
    tb = int(fr.info_np[v]["tile_base"])
    ok, ov, oe, orng = oracle.bin_sort(pv, cam, ocfg, tile_base=tb, val_base=v * n)
    s0 = int(touched[: v * n].astype(np.int64).sum())
    assert np.array_equal(tiles[s0:s0 + ok.size].astype(np.uint64), ok >> np.uint64(32))
    assert np.array_equal(vals[s0:s0 + ok.size], ov)
    # sampled tiles: the longest lists, random tiles, the ragged bottom row
    lk, lv, le, lr = oracle.bin_sort(pv, cam, ocfg)
    tx, ty = oracle.tiles_of(cam, ocfg)
    lens = lr[:, 1].astype(np.int64) - lr[:, 0]
    pick = np.unique(np.concatenate([np.argsort(lens)[-6:], rng.choice(tx * ty, n_tiles_sampled - 10, replace=False),
                                     np.arange((ty - 1) * tx, (ty - 1) * tx + 4)]))
    mask = np.zeros(tx * ty, np.uint8)
    mask[pick] = 1
    img, t32, _, nl = oracle.render(pv, lv, lr, cam, ocfg, tile_mask=mask)
    pix = np.zeros((cam.height, cam.width), bool)
    for t in pick:
        y0, x0 = (t // tx) * CFG["tile_h"], (t % tx) * CFG["tile_w"]
        pix[y0:y0 + CFG["tile_h"], x0:x0 + CFG["tile_w"]] = True
    assert_close_rel(view_slice(fr, res["image"], v)[:, pix], img[:, pix], 1e-5, 1e-3, f"image view {v}")
    assert np.array_equal(view_slice(fr, res["t_final"], v, 1)[pix].view(np.uint32), t32[pix].view(np.uint32))
    assert np.array_equal(view_slice(fr, res["n_last"], v, 1)[pix], nl[pix])
    d, i, idse, iimp = oracle.removal_effect(pv, lv, lr, cam, ocfg, tg[v], tile_mask=mask, per_instance=True)
    sel = np.concatenate([np.arange(lr[t, 0], lr[t, 1]) for t in pick]).astype(np.int64)
    slots = s0 + le[sel].astype(np.int64)
    _, imag = oracle.removal_magnitude(pv, lv, lr, cam, ocfg, tg[v], tile_mask=mask)
    assert_removal_close(res["inst_dse"][slots], idse[sel], imag[sel], f"tile partials view {v}")
    assert_close_abs_rel(res["inst_imp"][slots], iimp[sel], 1e-4, 1e-7, f"tile importance view {v}")
    assert np.count_nonzero(idse[sel]) > 200


def test_large_scene_in_8_view_chunks():
    """The 6M-splat scene's first 16 views of 1920x1080 run as the benchmark runs the large
    workload: two 8-view chunks sharing one buffer pool; view 9 (the second chunk's view 1)
    checked against the oracle."""
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    w = synth.workload("large")
    cams = w.cameras[:16]
    be = BatchedRemovalEffect(scene_to_device(w.scene), synth.cameras_to_array(cams), 8, **CFG)
    be.plan()
    tg = _targets(w.scene, cams, {9}, w.seed)
    flat = torch.from_numpy(np.concatenate([t.reshape(-1) for t in tg])).cuda()
    dmse = torch.zeros(w.scene.n, dtype=torch.float64, device="cuda")
    be.step(flat, dmse)  # both chunks, back to back on the pool; chunk 1 is resident afterwards
    fr = be.frames[1]
    res = frame_outputs(fr, pack_targets(fr, tg[8:16]), images=False)
    _check_view(fr, res, w.scene, cams[9], 1, tg[8:16], np.random.default_rng(9))
    assert np.count_nonzero(dmse.cpu().numpy()) > 0.1 * w.scene.n


def test_single_frame_of_300_1080p_views():
    """300 views of 1920x1080 in ONE frame (2,448,000 global tiles: keys with 22 tile bits, a
    three-pass tile partition) over a 100,000-splat scene of the large layout; views 0 and 299."""
    from gpu_util import build_frame

    sc = synth.ball_shell_scene(100_000, 1004, shell_outer=20.0)
    cams = synth.workload("large", n_override=1000).cameras
    assert len(cams) == 300
    fr = build_frame(sc, cams, **CFG)
    assert fr.total_tiles == 300 * 120 * 68 and fr.total_tiles >= 1 << 21
    tg = _targets(sc, cams, {0, 299}, 1004)
    res = frame_outputs(fr, pack_targets(fr, tg), images=False)
    rng = np.random.default_rng(299)
    for v in (0, 299):
        _check_view(fr, res, sc, cams[v], v, tg, rng)
