"""Pins of the gradient oracle (oracle/grad.py), no GPU.

* Its binary64 forward reproduces the C oracle's image (the two are independent restatements
  of Section 3's compositing; the C oracle rounds alpha to binary32, hence 1e-6).
* Its autograd gradient equals central finite differences of the C oracle's loss, for every
  parameter group, on a 200-splat 64x64 + 48x64 scene in a smooth configuration: alpha_min = 0,
  T_min = 0, alpha_max = 1 - 1e-6 (no threshold, stop or clamp can switch), squared-error loss
  (lambda = 1: the L1 term has a kink at c = c_t that finite differences cross), and only
  perturbations that leave every tile list and depth order unchanged.  Step h = 1e-3
  (2e-4 for means, whose truncation error is larger for sub-pixel splats); tolerance
  2e-3 relative plus the finite-difference noise floor of the binary32 decisions.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import grad as G


def test_binary64_forward_matches_c_oracle(tiny):
    cfg = oracle.make_config()
    cam = tiny.cameras[0]
    v = oracle.prepare_view(tiny.scene, cam, cfg)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
    tg = [(img + synth.target_noise(img.shape, 0.02, tiny.seed, 0)).astype(np.float32)]
    L, g, imgs = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, tg)
    assert np.max(np.abs(imgs[0] - img)) < 1e-5
    Lc, _ = G.oracle_loss(tiny.scene, tiny.cameras, cfg, tg)
    assert L == pytest.approx(Lc, rel=1e-6)
    for k in G.PARAM_KEYS:
        assert np.all(np.isfinite(g[k])) and np.count_nonzero(g[k]) > 0


def _same_order(a, b):
    return np.array_equal(a[1], b[1]) and np.array_equal(a[0] >> np.uint64(32), b[0] >> np.uint64(32))


def test_autograd_gradient_equals_finite_differences():
    cfg = oracle.make_config(alpha_min=0.0, t_min=0.0, alpha_max=1.0 - 1e-6)
    sc = synth.uniform_cube_scene(200, 31)
    cams = [synth.look_at_camera((0, 0, -3), 64, 64), synth.look_at_camera((2.0, 0.5, -2.2), 48, 64)]
    tg = []
    for v, c in enumerate(cams):
        pv = oracle.prepare_view(sc, c, cfg)
        im, *_ = oracle.render(pv, pv["vals"], pv["ranges"], c, cfg)
        tg.append((im + synth.target_noise(im.shape, 0.05, 5, v)).astype(np.float32))
    _, grad, _ = G.loss_and_grad(sc, cams, cfg, tg, lam=1.0)
    _, keys0 = G.oracle_loss(sc, cams, cfg, tg, lam=1.0)
    rng = np.random.default_rng(0)
    checked = {}
    for key in G.PARAM_KEYS:
        arr = getattr(sc, key)
        step = 2e-4 if key == "means" else 1e-3
        for _ in range(25):
            idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
            x0 = arr[idx]
            h = np.float32(step * max(1.0, abs(float(x0))))
            xp, xm = np.float32(x0 + h), np.float32(x0 - h)
            arr[idx] = xp
            lp, kp = G.oracle_loss(sc, cams, cfg, tg, lam=1.0)
            arr[idx] = xm
            lm, km = G.oracle_loss(sc, cams, cfg, tg, lam=1.0)
            arr[idx] = x0
            if not all(_same_order(a, c) and _same_order(b, c) for a, b, c in zip(kp, km, keys0)):
                continue
            fd = (lp - lm) / (float(xp) - float(xm))
            an = grad[key][idx]
            noise = 5e-9 * (1e-3 / step)
            assert abs(fd - an) <= 2e-3 * abs(an) + noise, (key, idx, fd, an)
            checked[key] = checked.get(key, 0) + 1
    assert all(checked.get(k, 0) >= 15 for k in G.PARAM_KEYS), checked
