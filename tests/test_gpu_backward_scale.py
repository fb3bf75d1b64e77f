"""Backward parity at full size: the 1M-splat, 8-view 1280x720 fine-tuning workload in the
launch configuration the benchmark times (all 8 views in one frame, 16x16 tiles, final
transmittance and n_last stored by the render), loss (1 - lambda) L1 + lambda L2 at lambda = 0.2.

The gradient oracle cannot differentiate the whole frame in seconds, so the loss is restricted
to sampled tiles: the device's dL/dc is set to zero outside 12 tiles of each of two views (the
four with the longest lists and eight random ones), which makes its parameter gradients those
of the loss summed over those pixels only, and the oracle differentiates the same restricted loss
(lists and image at those pixels, normalised by the whole frame's element count).  A pixel's
whole list is kept, so every splat that any sampled pixel composites gets its complete gradient
from those pixels.  Every element of every splat's gradient is compared: |gpu - oracle| <= 1e-4
|oracle| + KAPPA 2^-24 B, B the oracle's magnitude bound of the element (the tolerance of
tests/test_gpu_backward.py); splats that no sampled pixel composites must come out exactly 0.
Targets follow the workload's recipe (render + N(0, 0.01)); residuals within 1e-4 of zero are
moved to 1e-3 so that the L1 subgradient has the same sign on both sides.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import build_frame, oracle_cfg, pack_targets
from oracle import grad as G

pytestmark = pytest.mark.gpu

CFG = dict(tile_w=16, tile_h=16, batch=128)
VIEWS = (0, 5)
LONGEST, RANDOM = 4, 8
LAM = 0.2
REL, KAPPA = 1e-4, 4096.0
KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _tile_mask(cam, ranges, rng):
    """Pixels of the tiles with the LONGEST longest lists and of RANDOM other non-empty tiles."""
    tx_n = (cam.width + 15) // 16
    lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
    order = np.argsort(-lens, kind="stable")
    pick = list(order[:LONGEST])
    rest = np.setdiff1d(np.nonzero(lens > 0)[0], pick)
    pick += list(rng.choice(rest, size=RANDOM, replace=False))
    mask = np.zeros((cam.height, cam.width), bool)
    for t in pick:
        ty, tx = divmod(int(t), tx_n)
        mask[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = True
    return mask


def test_fullsize_backward_on_sampled_tiles():
    import torch

    w = synth.workload("grad")
    cams = w.cameras
    ocfg = oracle_cfg(CFG)
    rng = np.random.default_rng(17)
    targets, masks = [], []
    for v, cam in enumerate(cams):
        if v in VIEWS:
            pv = oracle.prepare_view(w.scene, cam, ocfg)
            img, *_ = oracle.render(pv, pv["vals"], pv["ranges"], cam, ocfg)
            tg = (img + synth.target_noise(img.shape, w.target_noise, w.seed, v)).astype(np.float32)
            near = np.abs(img - tg) < 1e-4
            tg[near] = (img[near] + 1e-3).astype(np.float32)
            targets.append(tg)
            masks.append(_tile_mask(cam, pv["ranges"], rng))
        else:
            targets.append(np.full((3, cam.height, cam.width), 0.3, np.float32))
            masks.append(np.zeros((cam.height, cam.width), bool))

    # device: the benchmark's frame, dL/dc restricted to the sampled pixels
    fr = build_frame(w.scene, cams, **CFG)
    img = fr.image_buffer()
    tf, nl = fr.pixel_buffer(), fr.pixel_buffer(torch.int32)
    fr.render(img, tf, nl)
    dL = torch.empty_like(img)
    loss = torch.zeros(1, dtype=torch.float64, device=img.device)
    fr.loss_grad(img, pack_targets(fr, targets), LAM, dL, loss)
    dL *= pack_targets(fr, [np.broadcast_to(m, (3,) + m.shape).astype(np.float32) for m in masks])
    grads = {k: torch.empty_like(fr.scene[k]) for k in KEYS}
    fr.render_backward(dL, grads, tf, nl)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    del fr, img, tf, nl, dL, grads
    torch.cuda.empty_cache()

    # oracle: the same restricted loss over the two views
    n_elems = sum(3 * c.pixels for c in cams)
    ocams = [cams[v] for v in VIEWS]
    otg = [targets[v] for v in VIEWS]
    om = [masks[v] for v in VIEWS]
    _, want, _ = G.loss_and_grad(w.scene, ocams, ocfg, otg, lam=LAM, masks=om, n_elems=n_elems)
    mag = G.loss_grad_magnitude(w.scene, ocams, ocfg, otg, lam=LAM, masks=om, n_elems=n_elems)

    eps = 2.0 ** -24
    n = w.scene.n
    reached = np.zeros(n, bool)  # splats some sampled pixel composites
    for k in KEYS:
        reached |= (mag[k].reshape(-1, n) > 0).any(axis=0)
    assert 1000 < reached.sum() < n // 2
    msgs = []
    for k in KEYS:
        g, o, b = got[k].reshape(-1), want[k].reshape(-1), mag[k].reshape(-1)
        assert np.all(np.isfinite(g)), f"{k}: non-finite gradient"
        err = np.abs(g - o)
        tol = REL * np.abs(o) + KAPPA * eps * b
        bad = err > tol
        seen = b > 0
        print(f"{k}: {int(seen.sum())} elements with terms; max |gpu - oracle| / (2^-24 B) = "
              f"{float(np.max(err[seen] / (eps * b[seen]))) if seen.any() else 0.0:.1f}")
        assert np.count_nonzero(o) > 100, f"{k}: too few elements reached by the sampled tiles"
        unreached = ~np.broadcast_to(reached, got[k].shape).reshape(-1)
        assert not np.any(g[unreached]), f"{k}: nonzero device gradient of a splat no sampled pixel composites"
        if bad.any():
            i = int(np.argmax(err - tol))
            msgs.append(f"{k}: {bad.sum()} of {bad.size} outside; worst got {g[i]!r} want {o[i]!r} B {b[i]!r}")
    assert not msgs, "\n".join(msgs)
