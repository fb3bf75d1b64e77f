"""Parity at full size: the 1M-splat, 16-view 1280x720 workload in the launch configuration
the benchmark times (all 16 views in one frame, 16x16 tiles, 128-splat batches).

The oracle cannot redo the whole frame in seconds, so it checks sampled outputs it can
compute one by one: preprocess and the complete binning/sort of two views (bit-exact), and
the render and removal effect of sampled tiles of those views (per-pixel image, T, n_last and
the per-(tile, splat) removal-effect partials).  Targets follow the workload's recipe.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (assert_close_abs_rel, assert_close_rel, assert_removal_close, build_frame,
                      check_against_whole_rect, frame_outputs, oracle_cfg, unpack_raster, view_slice)

pytestmark = pytest.mark.gpu

CFG = dict(tile_w=16, tile_h=16, batch=128)
VIEWS = (0, 11)


def oracle_targets(w, views):
    """Targets of the workload's recipe for the checked views -- the oracle's render of the scene
    with a seeded 5 % of the splats dropped, plus N(0, 0.01) noise -- and a flat grey image for
    the other views (their removal effects are not compared)."""
    ocfg = oracle_cfg(CFG)
    keep = synth.target_drop_mask(w.scene.n, w.target_drop, w.seed)
    sc2 = w.scene.subset(keep)
    out = []
    for v, c in enumerate(w.cameras):
        if v in views:
            pv = oracle.prepare_view(sc2, c, ocfg)
            img, *_ = oracle.render(pv, pv["vals"], pv["ranges"], c, ocfg)
            out.append((img + synth.target_noise(img.shape, w.target_noise, w.seed, v)).astype(np.float32))
        else:
            out.append(np.full((3, c.height, c.width), 0.3, np.float32))
    return out


@pytest.fixture(scope="module")
def big():
    import torch

    from gpu_util import pack_targets

    w = synth.workload("scene")
    fr = build_frame(w.scene, w.cameras, **CFG)
    tg = oracle_targets(w, VIEWS)
    res = frame_outputs(fr, pack_targets(fr, tg), images=False)
    r = unpack_raster(fr)
    m = fr.instance_count()
    tiles = fr.tiles[:m].cpu().numpy().view(np.uint32)
    vals = fr.vals[:m].cpu().numpy().view(np.uint32)
    touched = fr.touched.cpu().numpy().view(np.uint32)
    torch.cuda.synchronize()
    return w, fr, tg, res, r, tiles, vals, touched


def test_fullsize_preprocess_and_sort_views(big):
    w, fr, tg, res, r, tiles, vals, touched = big
    ocfg = oracle_cfg(CFG)
    act = oracle.activate(w.scene)
    n = w.scene.n
    counts = touched.reshape(len(w.cameras), n).astype(np.int64).sum(axis=1)
    for v in VIEWS:
        cam = w.cameras[v]
        pv = oracle.project(w.scene, act[0], cam, ocfg, act[1])
        assert np.array_equal(touched[v * n:(v + 1) * n], pv["touched"])
        vis = pv["touched"] > 0
        assert np.array_equal(r["mx"][v * n:(v + 1) * n][vis].view(np.uint32), pv["mean2d"][0][vis].view(np.uint32))
        assert np.array_equal(r["C"][v * n:(v + 1) * n][vis].view(np.uint32), pv["qcoef"][2][vis].view(np.uint32))
        tb = int(fr.info_np[v]["tile_base"])
        ok, ov, oe, orng = oracle.bin_sort(pv, cam, ocfg, tile_base=tb, val_base=v * n)
        s0 = int(counts[:v].sum())
        assert np.array_equal(tiles[s0:s0 + ok.size].astype(np.uint64), ok >> np.uint64(32))
        assert np.array_equal(vals[s0:s0 + ok.size], ov)


def test_fullsize_sampled_tiles(big):
    w, fr, tg, res, r, tiles, vals, touched = big
    ocfg = oracle_cfg(CFG)
    act = oracle.activate(w.scene)
    n = w.scene.n
    counts = touched.reshape(len(w.cameras), n).astype(np.int64).sum(axis=1)
    rng = np.random.default_rng(5)
    for v in VIEWS:
        cam = w.cameras[v]
        pv = oracle.project(w.scene, act[0], cam, ocfg, act[1])
        pv["opacity"] = act[1]
        ok, ov, oe, orng = oracle.bin_sort(pv, cam, ocfg)
        tx, ty = oracle.tiles_of(cam, ocfg)
        lens = orng[:, 1].astype(np.int64) - orng[:, 0]
        busy = np.argsort(lens)[-8:]  # the longest lists, plus random tiles and the ragged last row
        pick = np.unique(np.concatenate([busy, rng.choice(tx * ty, 12, replace=False),
                                         np.arange((ty - 1) * tx, (ty - 1) * tx + 4)]))
        mask = np.zeros(tx * ty, np.uint8)
        mask[pick] = 1
        img, t32, t64, nl = oracle.render(pv, ov, orng, cam, ocfg, tile_mask=mask)
        gimg = view_slice(fr, res["image"], v)
        gt = view_slice(fr, res["t_final"], v, 1)
        gnl = view_slice(fr, res["n_last"], v, 1)
        pix = np.zeros((cam.height, cam.width), bool)
        for t in pick:
            y0, x0 = (t // tx) * 16, (t % tx) * 16
            pix[y0:y0 + 16, x0:x0 + 16] = True
        assert_close_rel(gimg[:, pix], img[:, pix], 1e-5, 1e-3, f"image view {v}")
        assert np.array_equal(gt[pix].view(np.uint32), t32[pix].view(np.uint32))
        assert np.array_equal(gnl[pix], nl[pix])
        d, i, idse, iimp = oracle.removal_effect(pv, ov, orng, cam, ocfg, tg[v], tile_mask=mask, per_instance=True)
        sel = np.concatenate([np.arange(orng[t, 0], orng[t, 1]) for t in pick]).astype(np.int64)
        slots = int(counts[:v].sum()) + oe[sel].astype(np.int64)
        _, imag = oracle.removal_magnitude(pv, ov, orng, cam, ocfg, tg[v], tile_mask=mask)
        assert_removal_close(res["inst_dse"][slots], idse[sel], imag[sel], f"tile partials view {v}")
        assert_close_abs_rel(res["inst_imp"][slots], iimp[sel], 1e-4, 1e-7, f"tile importance view {v}")
        assert np.count_nonzero(idse[sel]) > 1000


def test_fullsize_culled_lists_against_whole_rectangle_binning(big):
    """Views 0 and 11 of the frame: every tile's device list is an order-preserving subsequence
    of the paper's footprint binning (all 3-sigma rectangle tiles, computed by the oracle with its
    tile test off) and holds every pair the oracle's walk of those lists composites; image,
    transmittance, last composited splat and per-view removal effects equal the oracle's from the
    whole-rectangle lists."""
    w, fr, tg, res, r, tiles, vals, touched = big
    dropped = check_against_whole_rect(fr, res, w.scene, w.cameras, CFG, VIEWS, tg)
    assert dropped > 0.2 * fr.instance_count() * len(VIEWS) / len(w.cameras)
