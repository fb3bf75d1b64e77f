"""Helpers shared by the GPU parity tests: run a frame through the C ABI, unpack buffers."""
from __future__ import annotations

import numpy as np

import oracle
import synth

RASTER_FIELDS = ("mx", "my", "A", "B", "C", "o", "pthr", "indefinite", "r", "g", "b", "rectw")
CULL_FIELDS = ("mask_lo", "mask_hi", "rectw2", "kept")


def oracle_cfg(cfg: dict):
    keep = {k: v for k, v in cfg.items() if k != "batch"}
    return oracle.make_config(**keep)


def build_frame(scene, cams, **cfg):
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    build.build()
    fr = RemovalEffectFrame(scene_to_device(scene), synth.cameras_to_array(cams), **cfg)
    fr.plan()
    torch.cuda.synchronize()
    return fr


def unpack_raster(fr) -> dict:
    r = fr.raster.cpu().numpy().reshape(-1, 12)
    cu = fr.cull.cpu().numpy().view(np.uint32).reshape(-1, 4)
    out = {k: r[:, i] for i, k in enumerate(RASTER_FIELDS)}
    out["rectw"] = out["rectw"].view(np.uint32)
    for i, k in enumerate(CULL_FIELDS):
        out[k] = cu[:, i]
    out["all_tiles"] = out["kept"] >> np.uint32(31)
    out["kept"] = out["kept"] & np.uint32(0x7FFFFFFF)
    out["mask"] = out["mask_lo"].astype(np.uint64) | (out["mask_hi"].astype(np.uint64) << np.uint64(32))
    return out


def frame_outputs(fr, targets_flat=None, importance=True, images=True):
    """Run render and (if targets given) removal effect; return numpy outputs."""
    import torch

    dev = fr.device
    img = fr.image_buffer()
    tfin = fr.pixel_buffer()
    nl = fr.pixel_buffer(torch.int32)
    fr.render(img, tfin, nl)
    out = dict(image=img, t_final=tfin, n_last=nl)
    if targets_flat is not None:
        dmse = torch.zeros(fr.n, dtype=torch.float64, device=dev)
        imp = torch.zeros(fr.n, dtype=torch.float64, device=dev) if importance else None
        dsse = torch.zeros(fr.n_views * fr.n, dtype=torch.float64, device=dev)
        img2 = fr.image_buffer() if images else None
        fr.removal_effect(targets_flat, dmse, imp, dsse_view=dsse, images=img2)
        out.update(dmse=dmse, importance=imp, dsse_view=dsse, image2=img2)
    torch.cuda.synchronize()
    res = {}
    for k, v in out.items():
        if v is None:
            res[k] = None
        else:
            res[k] = v.cpu().numpy()
    res["n_last"] = res["n_last"].view(np.uint32)
    res["inst_dse"] = fr.inst_dse[: fr.instance_count()].cpu().numpy()
    if fr.inst_imp is not None and targets_flat is not None and importance:
        res["inst_imp"] = fr.inst_imp[: fr.instance_count()].cpu().numpy()
    return res


def pack_targets(fr, targets):
    """list of [3, H, W] float32 arrays -> packed device buffer in frame layout."""
    import torch

    flat = np.concatenate([np.ascontiguousarray(t, np.float32).reshape(-1) for t in targets])
    assert flat.size == 3 * fr.total_pixels
    return torch.from_numpy(flat).to(fr.device)


def view_slice(fr, flat, v, planes=3):
    vi = fr.info_np[v]
    h, w, pb = int(vi["height"]), int(vi["width"]), int(vi["pixel_base"])
    if planes == 3:
        return flat[3 * pb: 3 * pb + 3 * h * w].reshape(3, h, w)
    return flat[pb: pb + h * w].reshape(h, w)


def assert_close_rel(got, want, rel, floor, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    tol = rel * np.maximum(np.abs(want), floor)
    bad = np.abs(got - want) > tol
    if bad.any():
        i = np.argmax(np.abs(got - want) - tol)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside tolerance; worst at {np.unravel_index(i, got.shape)}"
                             f" got {got.flat[i]!r} want {want.flat[i]!r}")


# Removal effects: |gpu - oracle| <= 1e-4 |oracle| + 1e-7 + KAPPA 2^-24 M, M the oracle's sum of the
# magnitudes of the terms each dSE is formed from (oracle.removal_magnitude).  The device forms
# every term in binary32 and recovers T_i by dividing the final T by (1 - alpha) back to front and
# the suffix S_> by adding the later splats' colours, one rounding per composited splat behind
# the entry, so a sum carries at most (chain length) 2^-24 M of rounding where terms cancel;
# KAPPA = 4096 covers chains of ~2000 composited splats per pixel.
KAPPA = 4096.0


def assert_removal_close(got, want, mag, what="", floor=1e-7):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    mag = np.asarray(mag, np.float64)
    err = np.abs(got - want)
    tol = 1e-4 * np.abs(want) + floor + KAPPA * 2.0 ** -24 * mag
    bad = err > tol
    seen = mag > 0
    worst = float(np.max(err[seen] / (2.0 ** -24 * mag[seen]))) if seen.any() else 0.0
    print(f"{what}: max |gpu - oracle| / (2^-24 M) = {worst:.1f}")
    if bad.any():
        i = int(np.argmax(err - tol))
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside tolerance; worst at {i}"
                             f" got {got.flat[i]!r} want {want.flat[i]!r} M {mag.flat[i]!r}")


def assert_close_abs_rel(got, want, rel, atol, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    tol = rel * np.abs(want) + atol
    bad = np.abs(got - want) > tol
    if bad.any():
        i = np.argmax(np.abs(got - want) - tol)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside tolerance; worst at {i}"
                             f" got {got.flat[i]!r} want {want.flat[i]!r}")


def check_against_whole_rect(fr, res, scene, cams, cfg, views, targets=None, act=None):
    """The device's (tile-culled) lists of the given views against the paper's plain footprint
    binning -- every tile of each splat's 3-sigma rectangle, no tile test -- as the oracle bins
    with its tile test switched off:

      * each tile's device list is an order-preserving subsequence of the whole-rectangle list;
      * it holds every (tile, splat) pair that the oracle's per-pixel walk of the
        whole-rectangle lists composites;
      * the device image equals the oracle's whole-rectangle render (image tolerance), the final
        transmittance bit for bit, and each pixel's last composited splat (n_last mapped through
        its list) is the same splat;
      * with targets, the per-view removal effects dSSE_k(v) equal the oracle's from the
        whole-rectangle lists (removal-effect tolerance).
    Returns the number of (tile, splat) pairs the culling dropped."""
    ocfg = oracle_cfg(cfg)
    n = scene.n
    if act is None:
        act = oracle.activate(scene)
    m = fr.instance_count()
    dvals = fr.vals[:m].cpu().numpy().view(np.uint32).astype(np.int64)
    dranges = fr.ranges.cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    dropped = 0
    for v in views:
        cam = cams[v]
        tw, th = cfg["tile_w"], cfg["tile_h"]
        tx, ty = oracle.tiles_of(cam, ocfg)
        pv = oracle.project(scene, act[0], cam, ocfg, act[1])
        pv["opacity"] = act[1]
        _, wv, _, wr = oracle.bin_sort(pv, cam, ocfg, whole_rect=True)
        wr = wr.astype(np.int64)
        tb = int(fr.info_np[v]["tile_base"])
        # (tile, splat) keys of both binnings, in list order
        wt = np.repeat(np.arange(tx * ty), wr[:, 1] - wr[:, 0])
        wkey = wt * n + wv.astype(np.int64)
        dr = dranges[tb:tb + tx * ty]
        dlen = np.maximum(dr[:, 1] - dr[:, 0], 0)
        didx = np.concatenate([np.arange(dr[t, 0], dr[t, 1]) for t in range(tx * ty) if dlen[t] > 0]
                              or [np.zeros(0, np.int64)])
        dt = np.repeat(np.arange(tx * ty), dlen)
        dk = dvals[didx] - v * n
        assert np.all((dk >= 0) & (dk < n)), f"view {v}: values outside the view"
        dkey = dt * n + dk
        order = np.argsort(wkey, kind="stable")
        at = np.searchsorted(wkey[order], dkey)
        assert np.all(at < wkey.size) and np.array_equal(wkey[order][np.minimum(at, wkey.size - 1)], dkey), \
            f"view {v}: a device pair is not in the whole-rectangle binning"
        wpos = order[at]  # position of each device pair in the whole-rectangle sorted list
        same = dt[1:] == dt[:-1]
        assert np.all(np.diff(wpos)[same] > 0), f"view {v}: device order differs from the whole-rectangle order"
        dropped += int(wkey.size - dkey.size)
        # every composited (tile, splat) pair of the whole-rectangle walk is in the device lists
        pix, ck, cpos = oracle.pixel_lists(pv, wv, wr.astype(np.uint32), cam, ocfg)
        ctile = (pix // cam.width) // th * tx + (pix % cam.width) // tw
        ckey = np.unique(ctile * n + ck.astype(np.int64))
        assert np.all(np.isin(ckey, dkey)), f"view {v}: a composited pair was culled"
        # render: image, T_final and the last composited splat of every pixel
        img, t32, t64, nl = oracle.render(pv, wv, wr.astype(np.uint32), cam, ocfg)
        assert_close_rel(view_slice(fr, res["image"], v), img, 1e-5, 1e-3, f"image view {v} (whole rectangles)")
        assert np.array_equal(view_slice(fr, res["t_final"], v, 1).view(np.uint32), t32.view(np.uint32))
        gnl = view_slice(fr, res["n_last"], v, 1).astype(np.int64)
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        tile = (ys // th) * tx + xs // tw
        gl = np.where(gnl > 0, dvals[np.clip(dr[tile, 0] + gnl - 1, 0, max(m - 1, 0))] - v * n, -1)
        wl = np.where(nl > 0, wv.astype(np.int64)[np.clip(wr[tile, 0] + nl.astype(np.int64) - 1, 0,
                                                          max(wv.size - 1, 0))], -1)
        assert np.array_equal(gl, wl), f"view {v}: last composited splat differs"
        if targets is not None:
            d, i = oracle.removal_effect(pv, wv, wr.astype(np.uint32), cam, ocfg, targets[v])
            mag, _ = oracle.removal_magnitude(pv, wv, wr.astype(np.uint32), cam, ocfg, targets[v])
            assert_removal_close(res["dsse_view"][v * n:(v + 1) * n], d, mag, f"dSSE view {v} (whole rectangles)")
    return dropped
