"""Non-finite splat parameters (injected on the host into the input tensors): potr_preprocess culls
every such splat in every view and reports POTR_ERR_NUMERIC with the count; everything else is
the result the oracle gives for the scene without those splats, and their removal effects,
importances and gradients are exactly 0."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (assert_close_rel, assert_removal_close, build_frame, frame_outputs, oracle_cfg, pack_targets,
                      view_slice)

pytestmark = pytest.mark.gpu

CFG = dict(tile_w=16, tile_h=16, batch=128)


def _poisoned():
    """5,000 splats in front of two cameras; six splats made non-finite in six ways: a NaN mean,
    an infinite log-scale, a NaN quaternion component, a -inf and a NaN opacity logit, and an
    infinite SH coefficient of a splat that both views see (so that its coefficients are read)."""
    sc = synth.uniform_cube_scene(5000, 77)
    cams = [synth.look_at_camera((0.0, 0.3, -3.0), 200, 150), synth.look_at_camera((2.5, -0.2, -1.5), 96, 160)]
    ocfg = oracle_cfg(CFG)
    seen = np.ones(sc.n, bool)
    for cam in cams:
        seen &= oracle.prepare_view(sc, cam, ocfg)["touched"] > 0
    sh_bad = int(np.nonzero(seen)[0][5])
    bad = np.array(sorted({10, 20, 30, 40, 50, sh_bad}))
    assert bad.size == 6
    sc.means[1, 10] = np.nan
    sc.log_scales[2, 20] = np.inf
    sc.quats[3, 30] = np.nan
    sc.opacity_logits[40] = -np.inf
    sc.opacity_logits[50] = np.nan
    sc.sh[5, 1, sh_bad] = np.inf
    return sc, cams, bad


def _clean_subset(sc, bad):
    keep = np.ones(sc.n, bool)
    keep[bad] = False
    return sc.subset(keep), keep


def test_nonfinite_splats_are_culled_and_reported():
    sc, cams, bad = _poisoned()
    clean, keep = _clean_subset(sc, bad)
    ocfg = oracle_cfg(CFG)
    fr = build_frame(sc, cams, **CFG)
    code, count = fr.nonfinite()
    assert code == oracle_status_numeric() and count == bad.size
    touched = fr.touched.cpu().numpy().view(np.uint32).reshape(len(cams), sc.n)
    assert np.all(touched[:, bad] == 0)
    # targets from the clean scene; the device's frame over the poisoned scene must match it
    tg = []
    ovs = []
    for v, cam in enumerate(cams):
        pv = oracle.prepare_view(clean, cam, ocfg)
        img, *_ = oracle.render(pv, pv["vals"], pv["ranges"], cam, ocfg)
        tg.append((img + synth.target_noise(img.shape, 0.02, 7, v)).astype(np.float32))
        ovs.append(pv)
    res = frame_outputs(fr, pack_targets(fr, tg))
    n_clean = clean.n
    for v, (cam, pv) in enumerate(zip(cams, ovs)):
        img, t32, _, _ = oracle.render(pv, pv["vals"], pv["ranges"], cam, ocfg)
        assert_close_rel(view_slice(fr, res["image"], v), img, 1e-5, 1e-3, f"image view {v}")
        assert np.array_equal(view_slice(fr, res["t_final"], v, 1).view(np.uint32), t32.view(np.uint32))
        d, i = oracle.removal_effect(pv, pv["vals"], pv["ranges"], cam, ocfg, tg[v])
        got = res["dsse_view"][v * sc.n:(v + 1) * sc.n]
        assert np.all(got[bad] == 0.0)
        mag, _ = oracle.removal_magnitude(pv, pv["vals"], pv["ranges"], cam, ocfg, tg[v])
        assert_removal_close(got[keep], d, mag, f"dSSE view {v}")
    assert np.all(res["dmse"][bad] == 0.0) and np.all(res["importance"][bad] == 0.0)
    assert np.all(np.isfinite(res["dmse"])) and np.all(np.isfinite(res["image"]))
    assert n_clean == sc.n - bad.size


def test_nonfinite_splats_get_zero_gradients():
    import torch

    sc, cams, bad = _poisoned()
    fr = build_frame(sc, cams, **CFG)
    img = fr.image_buffer()
    tf, nl = fr.pixel_buffer(), fr.pixel_buffer(torch.int32)
    fr.render(img, tf, nl)
    tg = img + 0.05
    dL = torch.empty_like(img)
    fr.loss_grad(img, tg, 0.2, dL)
    for store in (True, False):
        grads = {k: torch.full_like(fr.scene[k], 7.0) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        fr.render_backward(dL, grads, tf if store else None, nl if store else None)
        torch.cuda.synchronize()
        for k, g in grads.items():
            g = g.cpu().numpy()
            assert np.all(np.isfinite(g)), k
            assert np.all(g[..., bad] == 0.0), k
            assert np.count_nonzero(g) > 0, k


def oracle_status_numeric():
    from paper_2601_14821_gb300 import _binding as B

    return B.POTR_ERR_NUMERIC
