"""Batched removal effect over many view chunks (shared buffers, CUDA-graph replay) and the
autotuner; the 3M-splat, 200-view mixed-resolution workload checked on sampled outputs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_close_abs_rel, assert_removal_close, oracle_cfg

pytestmark = pytest.mark.gpu


def _mixed():
    sc = synth.uniform_cube_scene(5000, 77)
    cams = [synth.look_at_camera((0.0, 0.3, -3.0), 200, 150), synth.look_at_camera((2.5, -0.2, -1.5), 96, 160),
            synth.look_at_camera((-1.0, 0.0, 2.8), 128, 128), synth.look_at_camera((0.5, 2.0, 2.0), 64, 80)]
    return sc, cams


def _targets(sc, cams, seed):
    """Oracle render plus N(0, 0.02), the tiny workload's target recipe."""
    ocfg = oracle_cfg(dict(tile_w=16, tile_h=16))
    out = []
    for v, cam in enumerate(cams):
        pv = oracle.prepare_view(sc, cam, ocfg)
        img, *_ = oracle.render(pv, pv["vals"], pv["ranges"], cam, ocfg)
        out.append((img + synth.target_noise(img.shape, 0.02, seed, v)).astype(np.float32))
    return out


def test_chunking_and_graph_replay_give_the_same_bits():
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    sc, cams = _mixed()
    scene = scene_to_device(sc)
    rec = synth.cameras_to_array(cams)
    tg = _targets(sc, cams, 5)
    flat = torch.from_numpy(np.concatenate([t.reshape(-1) for t in tg])).cuda()
    results = []
    for vpc in (4, 3, 1):
        be = BatchedRemovalEffect(scene, rec, views_per_chunk=vpc, tile_w=16, tile_h=16, batch=256)
        be.plan()
        d = torch.zeros(sc.n, dtype=torch.float64, device="cuda")
        i = torch.zeros_like(d)
        be.step(flat, d, i)
        torch.cuda.synchronize()
        results.append((d.cpu().numpy(), i.cpu().numpy()))
        if vpc == 3:
            d2 = torch.zeros_like(d)
            i2 = torch.zeros_like(d)
            g = be.capture(flat, d2, i2)  # capture runs one warm-up pass eagerly
            d2.zero_()
            i2.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert np.array_equal(d2.cpu().numpy(), results[-1][0])
            assert np.array_equal(i2.cpu().numpy(), results[-1][1])
    for r in results[1:]:
        assert np.array_equal(r[0], results[0][0]) and np.array_equal(r[1], results[0][1])
    # and the oracle agrees on the whole thing
    ocfg = oracle_cfg(dict(tile_w=16, tile_h=16))
    want, wimp = oracle.dmse(sc, cams, ocfg, tg)
    mag = np.zeros(sc.n)
    for cam, t in zip(cams, tg):
        pv = oracle.prepare_view(sc, cam, ocfg)
        mag += oracle.removal_magnitude(pv, pv["vals"], pv["ranges"], cam, ocfg, t)[0] / (3.0 * cam.pixels) / len(cams)
    scale = 1.0 / (3.0 * min(c.pixels for c in cams))
    assert_removal_close(results[0][0], want, mag, "dMSE", floor=1e-7 * scale)
    assert_close_abs_rel(results[0][1], wimp, 1e-4, 1e-7 * scale, "importance")


def test_autotune_picks_a_timed_candidate():
    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.batched import SPLAT_BATCHES, TILE_SHAPES, autotune
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    sc, cams = _mixed()
    best = autotune(scene_to_device(sc), synth.cameras_to_array(cams), probe_views=4, steps=1, warmup=1)
    assert len(best["table"]) == len(TILE_SHAPES) * len(SPLAT_BATCHES)
    assert (best["tile_w"], best["tile_h"]) in TILE_SHAPES and best["batch"] in SPLAT_BATCHES
    assert best["ms_per_view"] == min(r["ms_per_view"] for r in best["table"])


def test_batched_workload_sampled_views_and_tiles():
    """3M splats, 200 views of mixed resolution, 16-view chunks as the benchmark runs them: the
    keys and values of one 1920x1080 and one 960x540 view bit-exact, and sampled tiles' removal
    partials, against the oracle."""
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    w = synth.workload("batched")
    cfg = dict(tile_w=16, tile_h=16, batch=256)
    rec = synth.cameras_to_array(w.cameras)
    be = BatchedRemovalEffect(scene_to_device(w.scene), rec, views_per_chunk=16, **cfg)
    be.plan()
    ocfg = oracle_cfg(cfg)
    act = oracle.activate(w.scene)
    n = w.scene.n
    sizes = [(c.width, c.height) for c in w.cameras]
    picks = [sizes.index((1920, 1080)), sizes.index((960, 540))]
    rng = np.random.default_rng(3)
    # Targets of the workload's recipe (render of the scene with 5 % of splats dropped, plus
    # N(0, 0.01)) on the tiles that are compared, a flat grey elsewhere.
    tg = [np.full((3, c.height, c.width), 0.3, np.float32) for c in w.cameras]
    keep = synth.target_drop_mask(n, w.target_drop, w.seed)
    sub = w.scene.subset(keep)
    masks = {}
    for v in picks:
        cam = w.cameras[v]
        tx, ty = oracle.tiles_of(cam, ocfg)
        pv = oracle.project(w.scene, act[0], cam, ocfg, act[1])
        lk, lvv, le, lr = oracle.bin_sort(pv, cam, ocfg)
        lens = lr[:, 1].astype(np.int64) - lr[:, 0]
        pick = np.unique(np.concatenate([np.argsort(lens)[-4:], rng.choice(tx * ty, 6, replace=False)]))
        mask = np.zeros(tx * ty, np.uint8)
        mask[pick] = 1
        masks[v] = (pick, mask)
        sv = oracle.prepare_view(sub, cam, ocfg)
        img, *_ = oracle.render(sv, sv["vals"], sv["ranges"], cam, ocfg, tile_mask=mask)
        noisy = (img + synth.target_noise(img.shape, w.target_noise, w.seed, v)).astype(np.float32)
        for t in pick:
            y0, x0 = (t // tx) * 16, (t % tx) * 16
            tg[v][:, y0:y0 + 16, x0:x0 + 16] = noisy[:, y0:y0 + 16, x0:x0 + 16]
    flat = torch.from_numpy(np.concatenate([t.reshape(-1) for t in tg])).cuda()
    for v in picks:
        ci, lv = divmod(v, be.views_per_chunk)
        fr = be.frames[ci]
        # run this chunk alone so its buffers hold its own keys and partials
        dm = torch.zeros(n, dtype=torch.float64, device="cuda")
        off = sum(f.total_pixels for f in be.frames[:ci])
        fr.step(flat[3 * off: 3 * (off + fr.total_pixels)], dm, torch.zeros_like(dm), n_views_total=len(w.cameras))
        torch.cuda.synchronize()
        cam = w.cameras[v]
        pv = oracle.project(w.scene, act[0], cam, ocfg, act[1])
        pv["opacity"] = act[1]
        touched = fr.touched.cpu().numpy().view(np.uint32).reshape(-1, n)
        start = int(touched[:lv].astype(np.int64).sum())
        tb = int(fr.info_np[lv]["tile_base"])
        ok, ov, oe, orng = oracle.bin_sort(pv, cam, ocfg, tile_base=tb, val_base=lv * n)
        tiles = fr.tiles[start:start + ok.size].cpu().numpy().view(np.uint32)
        vals = fr.vals[start:start + ok.size].cpu().numpy().view(np.uint32)
        assert np.array_equal(tiles.astype(np.uint64), ok >> np.uint64(32)) and np.array_equal(vals, ov)
        lk, lvv, le, lr = oracle.bin_sort(pv, cam, ocfg)
        pick, mask = masks[v]
        d, i, idse, iimp = oracle.removal_effect(pv, lvv, lr, cam, ocfg, tg[v], tile_mask=mask, per_instance=True)
        sel = np.concatenate([np.arange(lr[t, 0], lr[t, 1]) for t in pick]).astype(np.int64)
        got = fr.inst_dse[: fr.instance_count()].cpu().numpy()
        _, imag = oracle.removal_magnitude(pv, lvv, lr, cam, ocfg, tg[v], tile_mask=mask)
        assert_removal_close(got[start + le[sel].astype(np.int64)], idse[sel], imag[sel], f"tile partials view {v}")
        assert np.count_nonzero(idse[sel]) > 100
