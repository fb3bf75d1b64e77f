"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (fixed by the method's target, not tuned):
  * binning and sort (keys, values, ranges), tile rectangles, depth, the per-pair exponent
    coefficients, opacity, final transmittance and n_last: bit-exact;
  * rendered images: |gpu - oracle| <= 1e-5 max(|oracle|, 1e-3);
  * removal effects dSSE_k(v), importance and dMSE: |gpu - oracle| <= 1e-4 |oracle| + 1e-7,
    the absolute floor scaled by the same normalisation as the compared quantity;
  * SH colours (binary32 on the GPU, binary64 in the oracle): 2e-6 absolute.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (assert_close_abs_rel, assert_close_rel, assert_removal_close, build_frame,
                      check_against_whole_rect, frame_outputs, oracle_cfg, pack_targets, unpack_raster, view_slice)

pytestmark = pytest.mark.gpu

IMG_REL, IMG_FLOOR = 1e-5, 1e-3
DSE_REL, DSE_ABS = 1e-4, 1e-7


def _oracle_views(scene, cams, cfg):
    ocfg = oracle_cfg(cfg)
    act = oracle.activate(scene)
    out = []
    tile_base = 0
    for v, cam in enumerate(cams):
        pv = oracle.project(scene, act[0], cam, ocfg, act[1])
        pv["opacity"] = act[1]
        keys, vals, emit, ranges = oracle.bin_sort(pv, cam, ocfg, tile_base=tile_base, val_base=v * scene.n)
        pv.update(keys=keys, vals=vals, emit=emit, ranges=ranges, tile_base=tile_base)
        tx, ty = oracle.tiles_of(cam, ocfg)
        tile_base += tx * ty
        out.append(pv)
    return act, out


def _local_vals(pv, v, n):
    return (pv["vals"].astype(np.int64) - v * n).astype(np.uint32)


def _tiny_targets(scene, cams, cfg, seed):
    ocfg = oracle_cfg(cfg)
    act, ovs = _oracle_views(scene, cams, cfg)
    tg = []
    for v, (cam, pv) in enumerate(zip(cams, ovs)):
        img, *_ = oracle.render(pv, _local_vals(pv, v, scene.n), pv["ranges"], cam, ocfg)
        tg.append((img + synth.target_noise(img.shape, 0.02, seed, v)).astype(np.float32))
    return tg


MIXED = None


def mixed_workload():
    """5,000 splats, three views of ragged sizes (tails in both tile directions)."""
    global MIXED
    if MIXED is None:
        sc = synth.uniform_cube_scene(5000, 77)
        cams = [synth.look_at_camera((0.0, 0.3, -3.0), 200, 150), synth.look_at_camera((2.5, -0.2, -1.5), 96, 160),
                synth.look_at_camera((-1.0, 0.0, 2.8), 128, 128)]
        MIXED = (sc, cams)
    return MIXED


CFG16 = dict(tile_w=16, tile_h=16, batch=256)


@pytest.fixture(scope="module")
def tiny_run(tiny):
    cfg = CFG16
    fr = build_frame(tiny.scene, tiny.cameras, **cfg)
    tg = _tiny_targets(tiny.scene, tiny.cameras, cfg, tiny.seed)
    res = frame_outputs(fr, pack_targets(fr, tg))
    act, ovs = _oracle_views(tiny.scene, tiny.cameras, cfg)
    return fr, tg, res, act, ovs


def test_activation_bit_exact(tiny, tiny_run):
    fr, tg, res, act, ovs = tiny_run
    cov = fr.cov3d.cpu().numpy().reshape(6, -1)
    op = fr.opacity.cpu().numpy()
    assert np.array_equal(cov.view(np.uint32), act[0].view(np.uint32))
    assert np.array_equal(op.view(np.uint32), act[1].view(np.uint32))


def _check_preprocess(fr, scene, ovs):
    r = unpack_raster(fr)
    touched = fr.touched.cpu().numpy().view(np.uint32)
    rect = fr.rect.cpu().numpy().view(np.uint32).reshape(-1, 2)
    depth = fr.depth.cpu().numpy()
    n = scene.n
    for v, pv in enumerate(ovs):
        sl = slice(v * n, (v + 1) * n)
        assert np.array_equal(touched[sl], pv["touched"]), f"touched differs in view {v}"
        vis = pv["touched"] > 0
        g = {k: a[sl][vis] for k, a in r.items()}
        assert np.array_equal(depth[sl][vis].view(np.uint32), pv["depth"][vis].view(np.uint32))
        assert np.array_equal(g["mx"].view(np.uint32), pv["mean2d"][0][vis].view(np.uint32))
        assert np.array_equal(g["my"].view(np.uint32), pv["mean2d"][1][vis].view(np.uint32))
        for i, key in enumerate("ABC"):
            assert np.array_equal(g[key].view(np.uint32), pv["qcoef"][i][vis].view(np.uint32)), key
        rc = rect[sl][vis]
        x0, y0, x1, y1 = rc[:, 0] & 0xFFFF, rc[:, 0] >> 16, rc[:, 1] & 0xFFFF, rc[:, 1] >> 16
        for got, want in zip((x0, y0, x1, y1), pv["rect"][:, vis]):
            assert np.array_equal(got.astype(np.int64), want.astype(np.int64))
        rw = g["rectw"]
        assert np.array_equal(rw & 0x7FF, pv["rect"][0][vis]) and np.array_equal((rw >> 11) & 0x7FF, pv["rect"][1][vis])
        assert np.array_equal(rw >> 22, pv["rect"][2][vis] - pv["rect"][0][vis])
        for i, key in enumerate("rgb"):
            assert np.max(np.abs(g[key] - pv["rgb"][i][vis])) < 2e-6, key
        # kept-tile mask: the oracle's binned (tile, splat) pairs, as rectangle bit positions
        tx_n = int(fr.info_np[v]["tiles_x"])
        k = (pv["vals"].astype(np.int64) - v * n)
        t = (pv["keys"] >> np.uint64(32)).astype(np.int64) - pv["tile_base"]
        w = (pv["rect"][2] - pv["rect"][0]).astype(np.int64)
        area = w * (pv["rect"][3] - pv["rect"][1])
        pos = (t // tx_n - pv["rect"][1][k]) * w[k] + (t % tx_n - pv["rect"][0][k])
        small = area[k] <= oracle.CULL_MAX_TILES
        want = np.zeros(n, np.uint64)
        np.bitwise_or.at(want, k[small], np.left_shift(np.uint64(1), pos[small].astype(np.uint64)))
        big = area > oracle.CULL_MAX_TILES
        assert np.array_equal(g["all_tiles"], big[vis].astype(np.uint32))
        assert np.array_equal(g["mask"][~big[vis]], want[vis][~big[vis]])
        assert np.array_equal(g["rectw2"], rw) and np.array_equal(g["kept"], pv["touched"][vis])


def test_preprocess_bit_exact(tiny, tiny_run):
    fr, tg, res, act, ovs = tiny_run
    _check_preprocess(fr, tiny.scene, ovs)


def _check_binning(fr, ovs):
    m = fr.instance_count()
    tiles = fr.tiles[:m].cpu().numpy().view(np.uint32)
    vals = fr.vals[:m].cpu().numpy().view(np.uint32)
    ranges = fr.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2)
    okeys = np.concatenate([pv["keys"] for pv in ovs])
    ovals = np.concatenate([pv["vals"] for pv in ovs])
    assert m == okeys.size
    assert np.array_equal(tiles.astype(np.uint64), okeys >> np.uint64(32))
    assert np.array_equal(vals, ovals)
    start = 0
    for pv in ovs:
        rr = pv["ranges"].astype(np.int64)
        nonempty = rr[:, 1] > rr[:, 0]
        rr[nonempty] += start
        got = ranges[pv["tile_base"]: pv["tile_base"] + rr.shape[0]].astype(np.int64)
        assert np.array_equal(got[nonempty], rr[nonempty])
        assert np.all(got[~nonempty, 0] == got[~nonempty, 1])
        start += pv["keys"].size


def test_bin_sort_bit_exact(tiny, tiny_run):
    fr, tg, res, act, ovs = tiny_run
    _check_binning(fr, ovs)


def _check_render(fr, scene, cams, cfg, ovs, res):
    ocfg = oracle_cfg(cfg)
    for v, (cam, pv) in enumerate(zip(cams, ovs)):
        img, t32, t64, nl = oracle.render(pv, _local_vals(pv, v, scene.n), pv["ranges"], cam, ocfg)
        assert_close_rel(view_slice(fr, res["image"], v), img, IMG_REL, IMG_FLOOR, f"image view {v}")
        assert np.array_equal(view_slice(fr, res["t_final"], v, 1).view(np.uint32), t32.view(np.uint32))
        assert np.array_equal(view_slice(fr, res["n_last"], v, 1), nl)
        if res.get("image2") is not None:
            assert np.array_equal(res["image2"], res["image"])


def test_render_parity(tiny, tiny_run):
    fr, tg, res, act, ovs = tiny_run
    _check_render(fr, tiny.scene, tiny.cameras, CFG16, ovs, res)


def _check_removal(fr, scene, cams, cfg, ovs, res, targets):
    ocfg = oracle_cfg(cfg)
    n = scene.n
    dmse = np.zeros(n)
    imp = np.zeros(n)
    mag_dmse = np.zeros(n)
    for v, (cam, pv) in enumerate(zip(cams, ovs)):
        lv = _local_vals(pv, v, n)
        d, i, idse, iimp = oracle.removal_effect(pv, lv, pv["ranges"], cam, ocfg, targets[v], per_instance=True)
        mag, imag = oracle.removal_magnitude(pv, lv, pv["ranges"], cam, ocfg, targets[v])
        assert_removal_close(res["dsse_view"][v * n:(v + 1) * n], d, mag, f"dSSE view {v}")
        # per (tile, splat) partial sums, matched through the emission index
        base = int(sum(o["keys"].size for o in ovs[:v]))
        slots = base + pv["emit"].astype(np.int64)
        assert_removal_close(res["inst_dse"][slots], idse, imag, f"tile partials view {v}")
        if res.get("inst_imp") is not None:
            assert_close_abs_rel(res["inst_imp"][slots], iimp, DSE_REL, DSE_ABS, f"tile importance view {v}")
        dmse += d / (3.0 * cam.pixels) / len(cams)
        imp += i / float(cam.pixels) / len(cams)
        mag_dmse += mag / (3.0 * cam.pixels) / len(cams)
    scale = 1.0 / (3.0 * min(c.pixels for c in cams))
    assert_removal_close(res["dmse"], dmse, mag_dmse, "dMSE", floor=DSE_ABS * scale)
    if res.get("importance") is not None:
        assert_close_abs_rel(res["importance"], imp, DSE_REL, DSE_ABS * scale, "importance")
    assert np.count_nonzero(res["dmse"]) > 0.3 * n


def test_removal_effect_parity(tiny, tiny_run):
    fr, tg, res, act, ovs = tiny_run
    _check_removal(fr, tiny.scene, tiny.cameras, CFG16, ovs, res, tg)


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_mixed_views_every_tile_shape(tile):
    sc, cams = mixed_workload()
    cfg = dict(tile_w=tile[0], tile_h=tile[1], batch=128)
    fr = build_frame(sc, cams, **cfg)
    tg = _tiny_targets(sc, cams, cfg, 4242)
    res = frame_outputs(fr, pack_targets(fr, tg))
    act, ovs = _oracle_views(sc, cams, cfg)
    _check_preprocess(fr, sc, ovs)
    _check_binning(fr, ovs)
    _check_render(fr, sc, cams, cfg, ovs, res)
    _check_removal(fr, sc, cams, cfg, ovs, res, tg)


def test_culled_lists_against_whole_rectangle_binning_tiny(tiny, tiny_run):
    """The device's tile lists against the paper's footprint binning (every 3-sigma rectangle
    tile, the oracle's tile test off): order-preserving subsequences holding every composited
    pair, with the same image, transmittance, last composited splat and removal effects."""
    fr, tg, res, act, ovs = tiny_run
    dropped = check_against_whole_rect(fr, res, tiny.scene, tiny.cameras, CFG16, [0], tg, act)
    assert dropped > 0.1 * fr.instance_count()


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_culled_lists_against_whole_rectangle_binning_mixed(tile):
    sc, cams = mixed_workload()
    cfg = dict(tile_w=tile[0], tile_h=tile[1], batch=128)
    fr = build_frame(sc, cams, **cfg)
    tg = _tiny_targets(sc, cams, cfg, 4244)
    res = frame_outputs(fr, pack_targets(fr, tg))
    dropped = check_against_whole_rect(fr, res, sc, cams, cfg, range(len(cams)), tg)
    assert dropped > 0


def test_coincident_splats_keep_emission_order():
    """Splat 2j + 1 at splat 2j's position (equal depths, so equal (tile, depth) keys wherever
    both touch a tile): the device sort must keep such ties in emission order, as the oracle's
    stable sort does; binning bit-exact, render and removal effect within tolerance."""
    sc0, cams = mixed_workload()
    means = sc0.means.copy()
    means[:, 1::2] = means[:, 0:means.shape[1] - 1:2]
    sc = synth.Scene(means, sc0.log_scales, sc0.quats, sc0.opacity_logits, sc0.sh)
    cfg = dict(tile_w=16, tile_h=16, batch=128)
    fr = build_frame(sc, cams, **cfg)
    tg = _tiny_targets(sc, cams, cfg, 4243)
    res = frame_outputs(fr, pack_targets(fr, tg))
    act, ovs = _oracle_views(sc, cams, cfg)
    keys = np.concatenate([pv["keys"] for pv in ovs])
    assert np.count_nonzero(np.diff(keys.astype(np.int64)) == 0) > 1000
    _check_binning(fr, ovs)
    _check_render(fr, sc, cams, cfg, ovs, res)
    _check_removal(fr, sc, cams, cfg, ovs, res, tg)


def test_frame_over_65536_tiles_takes_three_tile_passes():
    """Nine 1920x1080 views (73,440 global tiles: 17 tile bits, three partition passes, the odd
    count that lands the result through the alternate buffer); binning, render and removal
    effect against the oracle."""
    sc = synth.uniform_cube_scene(4000, 91)
    cams = synth.ring_cameras(9, 3.0, 0.2, (1920, 1080))
    cfg = dict(tile_w=16, tile_h=16, batch=256)
    fr = build_frame(sc, cams, **cfg)
    assert fr.total_tiles > 65536
    tg = _tiny_targets(sc, cams, cfg, 91)
    res = frame_outputs(fr, pack_targets(fr, tg))
    act, ovs = _oracle_views(sc, cams, cfg)
    _check_binning(fr, ovs)
    _check_render(fr, sc, cams, cfg, ovs, res)
    _check_removal(fr, sc, cams, cfg, ovs, res, tg)


def test_batch_size_and_view_chunking_do_not_change_bits():
    sc, cams = mixed_workload()
    outs = []
    for batch in (128, 256, 512):
        fr = build_frame(sc, cams, tile_w=16, tile_h=16, batch=batch)
        tg = _tiny_targets(sc, cams, dict(tile_w=16, tile_h=16), 9)
        outs.append(frame_outputs(fr, pack_targets(fr, tg)))
    for o in outs[1:]:
        for k in ("image", "t_final", "n_last", "dmse", "importance", "dsse_view", "inst_dse"):
            assert np.array_equal(o[k], outs[0][k]), k
    # one view per frame, views added in order, equals the whole frame bit for bit
    import torch

    dmse = torch.zeros(sc.n, dtype=torch.float64, device="cuda")
    imp = torch.zeros(sc.n, dtype=torch.float64, device="cuda")
    for v, cam in enumerate(cams):
        fr = build_frame(sc, [cam], tile_w=16, tile_h=16, batch=256)
        fr.removal_effect(pack_targets(fr, [tg[v]]), dmse, imp, n_views_total=len(cams))
    torch.cuda.synchronize()
    assert np.array_equal(dmse.cpu().numpy(), outs[0]["dmse"])
    assert np.array_equal(imp.cpu().numpy(), outs[0]["importance"])


def test_repeat_runs_are_bit_identical(tiny, tiny_run):
    fr, tg, res, act, ovs = tiny_run
    res2 = frame_outputs(fr, pack_targets(fr, tg))
    for k in ("image", "t_final", "n_last", "dmse", "importance", "dsse_view", "inst_dse"):
        assert np.array_equal(res2[k], res[k]), k


def test_capacity_overflow_is_reported_and_safe(tiny):
    import torch

    from paper_2601_14821_gb300 import POTR_ERR_CAPACITY

    fr = build_frame(tiny.scene, tiny.cameras, **CFG16)
    m = fr.instance_count()
    fr._alloc(m // 2)
    fr.bin_sort()
    torch.cuda.synchronize()
    code, need = fr.status.tolist()
    assert code == POTR_ERR_CAPACITY and need == m
    ranges = fr.ranges.cpu().numpy()
    assert np.all(ranges == 0)
    dmse = torch.zeros(fr.n, dtype=torch.float64, device="cuda")
    fr.removal_effect(pack_targets(fr, [np.zeros((3, 128, 128), np.float32)]), dmse)
    torch.cuda.synchronize()
    assert np.all(dmse.cpu().numpy() == 0)


def test_everything_culled_gives_empty_frame(tiny):
    cam = synth.look_at_camera((0.0, 0.0, -30.0), 64, 48)
    cam.w2c[8:11] *= -1.0  # look away from the scene: every splat is behind the camera
    cam.w2c[11] = -cam.w2c[11]
    fr = build_frame(tiny.scene, [cam], **CFG16)
    assert fr.instance_count() == 0
    res = frame_outputs(fr, pack_targets(fr, [np.full((3, 48, 64), 0.5, np.float32)]))
    assert np.all(res["image"] == 0) and np.all(res["t_final"] == 1) and np.all(res["n_last"] == 0)
    assert np.all(res["dmse"] == 0)


def test_single_splat_closed_form():
    """One splat on the optical axis: dSE = PD (PD + 2 (c - c_t)) with PD = -alpha c_0, so the
    GPU result must equal the oracle's and alpha c0 (alpha c0 - 2 (alpha c0 - c_t)) summed."""
    means = np.zeros((3, 1), np.float32)
    sh = np.zeros((16, 3, 1), np.float32)
    sh[0, :, 0] = [0.8, 0.1, -0.4]
    sc = synth.Scene(means, np.full((3, 1), -2.5, np.float32), np.array([[1.0], [0], [0], [0]], np.float32),
                     np.array([2.0], np.float32), sh)
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 80, 72)
    cfg = dict(tile_w=16, tile_h=16, batch=128)
    fr = build_frame(sc, [cam], **cfg)
    tg = [np.full((3, 72, 80), 0.25, np.float32)]
    res = frame_outputs(fr, pack_targets(fr, tg))
    act, ovs = _oracle_views(sc, [cam], cfg)
    _check_removal(fr, sc, [cam], cfg, ovs, res, tg)
    img = view_slice(fr, res["image"], 0).astype(np.float64)
    want = np.sum(img * (img - 2.0 * (img - 0.25)))
    assert res["dsse_view"][0] == pytest.approx(want, rel=1e-5)


def test_tile_schedule_is_a_longest_first_permutation_and_changes_no_bit():
    import torch

    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    sc, cams = mixed_workload()
    tg = _tiny_targets(sc, cams, CFG16, 31)
    outs = []
    for sched in (False, True):
        fr = RemovalEffectFrame(scene_to_device(sc), synth.cameras_to_array(cams), schedule=sched, **CFG16)
        fr.plan()
        outs.append(frame_outputs(fr, pack_targets(fr, tg)))
        if sched:
            torch.cuda.synchronize()
            order = fr.order.cpu().numpy().view(np.uint32)[: fr.total_tiles]
            assert np.array_equal(np.sort(order), np.arange(fr.total_tiles, dtype=np.uint32))
            r = fr.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
            lens = (r[:, 1] - r[:, 0])[order]
            bucket = np.where(lens == 0, 0, np.floor(np.log2(np.maximum(lens, 1))).astype(np.int64) + 1)
            assert np.all(np.diff(bucket) <= 0)
    for k in ("image", "t_final", "n_last", "dmse", "importance", "dsse_view", "inst_dse"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_bounded_wait_times_out_and_reports():
    """The sort's look-back gives up on a predecessor that never publishes: it writes
    POTR_ERR_TIMEOUT to the status word and returns; the context keeps working."""
    import torch

    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300 import build

    build.build()
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    status = torch.zeros(2, dtype=torch.int64, device="cuda")
    B.potr_selftest_wait_timeout(ws, 1000, status)
    torch.cuda.synchronize()
    assert int(status[0].item()) == B.POTR_ERR_TIMEOUT
    fr = build_frame(*mixed_workload(), **CFG16)  # the device is still usable afterwards
    assert fr.instance_count() > 0


def test_per_splat_reduce_over_many_views_and_long_runs():
    """The per-splat reduce against binary64 sums of the device's own instance partials, on a
    frame of 70 views (the views as one pipelined sequence, past 64) whose splats are large
    enough (about 6 x 6 tiles each) that a warp's 32 splats hold more than 256 slots in a view,
    so their runs are staged in several chunks.  dSSE_k(v), dMSE_k and I_k must match those sums
    within the rounding of binary32 view sums and terms: 1e-6 of the sums of magnitudes."""
    import torch

    sc = synth.uniform_cube_scene(4000, 77)
    sc.log_scales = (sc.log_scales + 2.5).astype(np.float32)
    cams = synth.ring_cameras(70, 3.5, 0.5, (320, 240))
    fr = build_frame(sc, cams, **CFG16)
    tg = [np.full((3, c.height, c.width), 0.3, np.float32) for c in cams]
    res = frame_outputs(fr, pack_targets(fr, tg), images=False)
    n, nv = sc.n, len(cams)
    touched = fr.touched.cpu().numpy().view(np.uint32).astype(np.int64)
    offsets = fr.offsets.cpu().numpy().view(np.uint32).astype(np.int64)
    P = np.array([c.width * c.height for c in cams], np.float64)

    nz = touched > 0

    def view_sums(x):  # each (view, splat)'s run of slots, summed on its own in binary64
        out = np.zeros(nv * n)
        out[nz] = np.add.reduceat(x.astype(np.float64), offsets[nz])  # runs are contiguous, in vk order
        return out.reshape(nv, n)

    s_d, a_d = view_sums(res["inst_dse"]), view_sums(np.abs(res["inst_dse"]))
    s_i, a_i = view_sums(res["inst_imp"]), view_sums(np.abs(res["inst_imp"]))
    runs = np.add.reduceat(touched.reshape(nv, n), np.arange(0, n, 32), axis=1)
    assert runs.max() > 256 and (runs > 256).sum() > 100  # many warps stage more than one chunk
    assert np.count_nonzero(s_d) > 0.2 * s_d.size  # large splats hide many others
    err = np.abs(res["dsse_view"].reshape(nv, n) - s_d)
    assert np.all(err <= 1e-6 * a_d), float(np.max(err - 1e-6 * a_d))
    w = 1.0 / (P[:, None] * nv)
    want_d, mag_d = (s_d * w / 3.0).sum(axis=0), (a_d * w / 3.0).sum(axis=0)
    want_i, mag_i = (s_i * w).sum(axis=0), (a_i * w).sum(axis=0)
    assert np.all(np.abs(res["dmse"] - want_d) <= 1e-6 * mag_d)
    assert np.all(np.abs(res["importance"] - want_i) <= 1e-6 * mag_i)
    del fr
    torch.cuda.empty_cache()
