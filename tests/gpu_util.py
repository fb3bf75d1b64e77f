"""Helpers shared by the GPU parity tests: run a frame through the C ABI, unpack buffers."""
from __future__ import annotations

import numpy as np

import oracle
import synth

RASTER_FIELDS = ("mx", "my", "A", "B", "C", "o", "pthr", "zero", "r", "g", "b", "rectw")
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


def assert_close_abs_rel(got, want, rel, atol, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    tol = rel * np.abs(want) + atol
    bad = np.abs(got - want) > tol
    if bad.any():
        i = np.argmax(np.abs(got - want) - tol)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} outside tolerance; worst at {i}"
                             f" got {got.flat[i]!r} want {want.flat[i]!r}")
