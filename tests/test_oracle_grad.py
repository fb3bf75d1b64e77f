"""Pins of the gradient oracle (oracle/grad.py), no GPU.

* Its binary64 forward reproduces the C oracle's image (the two are independent restatements
  of Section 3's compositing; the C oracle rounds alpha to binary32, hence 1e-6).
* Its autograd gradient equals central finite differences of the C oracle's loss, for every
  parameter group, on a 200-splat 64x64 + 48x64 scene in a smooth configuration: alpha_min = 0,
  T_min = 0, alpha_max = 1 - 1e-6 (no threshold, stop or clamp can switch), squared-error loss
  (lambda = 1: the L1 term has a kink at c = c_t that finite differences cross), and only
  perturbations that leave every tile list and depth order unchanged.  Step h = 1e-3
  (2e-4 for means, whose truncation error is larger for sub-pixel splats); tolerance
  2e-3 relative plus the finite-difference noise floor of the binary32 decisions.  Again at
  lambda = 0.2 with every residual kept positive, so that the L1 term's weight enters.
* The loss in closed form when every residual is delta: (1 - lambda) |delta| + lambda delta^2.
* A zero residual (targets equal to the render) gives a loss and gradients of exactly 0.
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


def _smooth_setup(offset=None):
    """200 splats seen by a 64x64 and a 48x64 view, with no threshold, stop or clamp that a small
    perturbation can switch; targets are the render plus noise, or minus ``offset`` (a residual
    of one sign everywhere)."""
    cfg = oracle.make_config(alpha_min=0.0, t_min=0.0, alpha_max=1.0 - 1e-6)
    sc = synth.uniform_cube_scene(200, 31)
    cams = [synth.look_at_camera((0, 0, -3), 64, 64), synth.look_at_camera((2.0, 0.5, -2.2), 48, 64)]
    tg = []
    for v, c in enumerate(cams):
        pv = oracle.prepare_view(sc, c, cfg)
        im, *_ = oracle.render(pv, pv["vals"], pv["ranges"], c, cfg)
        if offset is None:
            tg.append((im + synth.target_noise(im.shape, 0.05, 5, v)).astype(np.float32))
        else:
            tg.append(im - offset)
    return cfg, sc, cams, tg


def _finite_difference_check(cfg, sc, cams, tg, lam, samples, need, seed=0, noise_scale=1.0):
    # The C oracle's binary32 alphas put a noise floor on the difference quotient proportional to
    # |dL/dc|: about 2 |r| ~ 0.1 for squared error on 0.05 noise, the unit of noise_scale.
    _, grad, _ = G.loss_and_grad(sc, cams, cfg, tg, lam=lam)
    _, keys0 = G.oracle_loss(sc, cams, cfg, tg, lam=lam)
    rng = np.random.default_rng(seed)
    checked = {}
    for key in G.PARAM_KEYS:
        arr = getattr(sc, key)
        step = 2e-4 if key == "means" else 1e-3
        for _ in range(samples):
            idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
            x0 = arr[idx]
            h = np.float32(step * max(1.0, abs(float(x0))))
            xp, xm = np.float32(x0 + h), np.float32(x0 - h)
            arr[idx] = xp
            lp, kp = G.oracle_loss(sc, cams, cfg, tg, lam=lam)
            arr[idx] = xm
            lm, km = G.oracle_loss(sc, cams, cfg, tg, lam=lam)
            arr[idx] = x0
            if not all(_same_order(a, c) and _same_order(b, c) for a, b, c in zip(kp, km, keys0)):
                continue
            fd = (lp - lm) / (float(xp) - float(xm))
            an = grad[key][idx]
            noise = 5e-9 * (1e-3 / step) * noise_scale
            assert abs(fd - an) <= 2e-3 * abs(an) + noise, (key, idx, fd, an)
            checked[key] = checked.get(key, 0) + 1
    assert all(checked.get(k, 0) >= need for k in G.PARAM_KEYS), checked


def test_autograd_gradient_equals_finite_differences():
    _finite_difference_check(*_smooth_setup(), lam=1.0, samples=25, need=15)


def test_mixed_loss_gradient_equals_finite_differences():
    """lambda = 0.2 (both terms): targets 0.5 below the render keep every residual positive, so
    the L1 term is smooth under the perturbations and its weight 1 - lambda is exercised.
    |dL/dc| = (1 - lambda) + 2 lambda r = 1.0, ten times the squared-error setup's, and so is the
    finite-difference noise floor."""
    _finite_difference_check(*_smooth_setup(offset=0.5), lam=0.2, samples=10, need=6, seed=1, noise_scale=10.0)


@pytest.mark.parametrize("delta", [0.25, -0.125])
def test_loss_closed_form_for_a_constant_residual(delta):
    """With every target delta below the render, each of the 3 x (64 x 64 + 48 x 64) residuals is
    delta and the loss is (1 - lambda) |delta| + lambda delta^2 for any lambda: pins the weights
    of the two terms and the mean over channels, pixels and views of unequal sizes."""
    cfg, sc, cams, tg = _smooth_setup(offset=delta)
    for lam in (0.0, 0.2, 1.0):
        want = (1.0 - lam) * abs(delta) + lam * delta * delta
        L, _ = G.oracle_loss(sc, cams, cfg, tg, lam=lam)
        assert L == pytest.approx(want, abs=1e-12)
        Lg, _, _ = G.loss_and_grad(sc, cams, cfg, tg, lam=lam)
        assert Lg == pytest.approx(want, abs=2e-5)  # binary64 alphas against the C oracle's binary32


def test_zero_residual_gives_zero_gradient(tiny):
    """Targets equal to the oracle's own binary64 render: every residual is exactly 0, where the
    L1 term's subgradient is 0 (sign 0 = 0), so the loss and every gradient are exactly 0."""
    cfg = oracle.make_config()
    first = []
    for cam in tiny.cameras:
        v = oracle.prepare_view(tiny.scene, cam, cfg)
        img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
        first.append(np.zeros_like(img))
    _, _, imgs = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, first)
    for lam in (0.0, 0.2):
        L, g, _ = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, [np.asarray(i, np.float64) for i in imgs], lam=lam)
        assert L == 0.0
        for k in G.PARAM_KEYS:
            assert np.count_nonzero(g[k]) == 0, (lam, k)


def test_binary64_forward_matches_c_oracle_at_the_clamps():
    """A scene that reaches every clamp of the forward: large splats beyond the Jacobian clamp
    whose footprints reach into the image, opaque splats (alpha clamped to alpha_max) and splats
    whose colour clamps at 0.  The binary64 forward still reproduces the C oracle's image."""
    from scenes import clamp_scene

    cfg = oracle.make_config()
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 64, 64)
    sc, m = clamp_scene(cam)
    W = cam.w2c.reshape(3, 4).astype(np.float64)
    lim = 1.3 * 0.5 * cam.width / cam.fx
    act = oracle.activate(sc)
    v = oracle.prepare_view(sc, cam, cfg, act)
    n = sc.n
    assert np.all(v["touched"][n - m:] > 0)
    t = (W[:, :3] @ sc.means[:, n - m:].astype(np.float64) + W[:, 3:4])
    assert np.all(np.abs(t[0] / t[2]) > lim)
    assert np.all(v["rgb"][0, 40:80] == 0.0) and np.all(act[1][:40] > 0.999)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
    keep = np.ones(n, bool)
    keep[n - m:] = False
    v2 = oracle.prepare_view(sc.subset(keep), cam, cfg)
    img2, *_ = oracle.render(v2, v2["vals"], v2["ranges"], cam, cfg)
    assert np.max(np.abs(img - img2)) > 0.05  # the splats beyond the clamp show in the image
    _, _, imgs = G.loss_and_grad(sc, [cam], cfg, [np.zeros_like(img)])
    assert np.max(np.abs(imgs[0] - img)) < 1e-5


# ------------------------------------------------------------------------------------------
# the per-element magnitude bound used as the device gradients' rounding scale
# ------------------------------------------------------------------------------------------

def test_gradient_magnitude_bounds_every_gradient_element():
    """B_p (sum over entries of magnitudes, loss_grad_magnitude) is at least |dL/dp| for every
    element, for the squared-error loss and at lambda = 0.2, and is reached with equality by some
    elements (a sum of terms of one sign)."""
    sc = synth.uniform_cube_scene(200, 88)
    cam = synth.look_at_camera((0.0, 0.3, -3.0), 64, 64)
    cfg = oracle.make_config()
    v = oracle.prepare_view(sc, cam, cfg)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
    tg = [(img + synth.target_noise(img.shape, 0.02, 3, 0)).astype(np.float32)]
    for lam in (1.0, 0.2):
        _, g, _ = G.loss_and_grad(sc, [cam], cfg, tg, lam=lam)
        B = G.loss_grad_magnitude(sc, [cam], cfg, tg, lam=lam)
        for k in G.PARAM_KEYS:
            assert np.all(B[k] >= np.abs(g[k]) * (1.0 - 1e-12)), k
            assert np.count_nonzero(B[k]) > 0.5 * B[k].size, k
        # an SH coefficient of a splat seen in one view gets its gradient only through the colour
        assert np.max(np.abs(g["sh"]) / np.maximum(B["sh"], 1e-300)) > 1.0 - 1e-9


def _two_splats_one_pixel():
    """A 1 x 1 image and two splats on the optical axis (front at z = 2, back at z = 3) wide
    enough that the pixel centre sees both at their peaks (G = 1, alpha = o)."""
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 1, 1)
    means = np.array([[0.0, 0.0], [0.0, 0.0], [-1.0, 0.0]], np.float32)
    sh = np.zeros((16, 3, 2), np.float32)
    sh[0, :, 0] = [0.9, 0.2, -0.3]
    sh[0, :, 1] = [-0.1, 0.6, 0.4]
    sc = synth.Scene(means, np.full((3, 2), -1.0, np.float32), np.array([[1.0, 1.0], [0, 0], [0, 0], [0, 0]], np.float32),
                     np.array([0.3, -0.2], np.float32), sh)
    return sc, cam


def test_gradient_magnitude_closed_form_two_splats():
    """Two splats composited at one pixel (front 0, back 1, alpha_i = o_i, T_0 = 1, T_1 = 1 - a0,
    c = a0 c0 + (1 - a0) a1 c1, g = dL/dc = 2 (c - c_t) / 3):
      dL/dlogit_0 = a0 (1 - o0) sum_ch g (c0 - a1 c1)   and its bound  a0 (1 - o0) sum_ch |g| (c0 + a1 c1),
      dL/dlogit_1 = a1 (1 - o1) (1 - a0) sum_ch g c1     bound the same in |g|,
      dL/dDC_0,ch = g_ch a0 Y_0                          bound |g_ch| a0 Y_0.
    The suffix of the front splat's alpha adjoint enters the bound with a plus sign."""
    sc, cam = _two_splats_one_pixel()
    cfg = oracle.make_config()
    tg = [np.full((3, 1, 1), 0.2, np.float32)]
    _, g, imgs = G.loss_and_grad(sc, [cam], cfg, tg, lam=1.0)
    B = G.loss_grad_magnitude(sc, [cam], cfg, tg, lam=1.0)
    o = 1.0 / (1.0 + np.exp(-sc.opacity_logits.astype(np.float64)))
    a0, a1 = o
    Y0 = 0.5 / np.sqrt(np.pi)
    c0 = np.maximum(sc.sh[0, :, 0].astype(np.float64) * Y0 + 0.5, 0.0)
    c1 = np.maximum(sc.sh[0, :, 1].astype(np.float64) * Y0 + 0.5, 0.0)
    c = a0 * c0 + (1.0 - a0) * a1 * c1
    assert np.allclose(imgs[0].reshape(3), c, rtol=1e-6)
    gc = 2.0 * (c - 0.2) / 3.0
    assert g["opacity_logits"][0] == pytest.approx(a0 * (1 - a0) * np.sum(gc * (c0 - a1 * c1)), rel=1e-6)
    assert B["opacity_logits"][0] == pytest.approx(a0 * (1 - a0) * np.sum(np.abs(gc) * (c0 + a1 * c1)), rel=1e-6)
    want1 = a1 * (1 - a1) * (1 - a0) * np.sum(np.abs(gc) * c1)
    assert B["opacity_logits"][1] == pytest.approx(want1, rel=1e-6)
    assert abs(g["opacity_logits"][1]) == pytest.approx(want1, rel=1e-6)
    assert np.allclose(B["sh"][0, :, 0], np.abs(gc) * a0 * Y0, rtol=1e-6)
    assert np.allclose(np.abs(g["sh"][0, :, 0]), B["sh"][0, :, 0], rtol=1e-9)


def _screen(sc, cam, cfg, tg, lam):
    import torch

    p = G.to_params(sc, requires_grad=False)
    sigma, o = G.activate(p)
    pr = G.project(p, sigma, cam, cfg)
    pr = {k: v.detach() for k, v in pr.items()}
    pr["o"] = o.detach()
    v = oracle.prepare_view(sc, cam, cfg)
    pix, k, _ = oracle.pixel_lists(v, v["vals"], v["ranges"], cam, cfg)
    n_elems = 3 * cam.pixels
    return (G.screen_magnitudes(pr, cam, cfg, tg, lam, n_elems, pix, k).numpy(),
            G.screen_grad(pr, cam, cfg, tg, lam, n_elems, pix, k).numpy(), torch)


def test_screen_magnitudes_bound_the_screen_gradients():
    """Per splat and screen quantity (centre, conic, opacity, colour) the magnitude sum bounds the
    autograd gradient of the loss with respect to that quantity, on a 200-splat view."""
    sc = synth.uniform_cube_scene(200, 88)
    cam = synth.look_at_camera((0.0, 0.3, -3.0), 64, 64)
    cfg = oracle.make_config()
    v = oracle.prepare_view(sc, cam, cfg)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
    tg = (img + synth.target_noise(img.shape, 0.02, 3, 0)).astype(np.float32)
    for lam in (1.0, 0.2):
        Gm, Gr, _ = _screen(sc, cam, cfg, tg, lam)
        assert np.all(Gm >= np.abs(Gr) * (1.0 - 1e-12))
        assert np.count_nonzero(Gm[:, 0]) > 50


def test_screen_magnitudes_equal_the_gradient_without_cancellation():
    """One splat at one pixel (a 1 x 1 image), its centre off the pixel centre along a diagonal
    where the conic's cross term has the sign of the diagonal terms, every channel above its
    target: each screen quantity's gradient is a single product of terms of one sign, so the
    magnitude sums equal its absolute value exactly (centre terms |ca dx| + |cb dy| added,
    opacity through exp(power))."""
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 1, 1)
    sh = np.zeros((16, 3, 1), np.float32)
    sh[0, :, 0] = [0.9, 0.4, 0.7]
    q = np.array([[np.cos(0.3)], [0.0], [0.0], [np.sin(0.3)]], np.float32)  # rotation about z: cb != 0
    cfg = oracle.make_config()
    tg = np.zeros((3, 1, 1), np.float32)

    def scene(ox, oy):
        return synth.Scene(np.array([[ox], [oy], [0.0]], np.float32), np.array([[-1.2], [-2.0], [-1.5]], np.float32),
                           q, np.array([0.4], np.float32), sh)

    # pick the centre offset whose pixel offsets (dx, dy) have sign(dx) sign(dy) = sign(cb)
    for ox, oy in [(4e-4, 3e-4), (4e-4, -3e-4)]:
        sc = scene(ox, oy)
        pr = G.project(G.to_params(sc, requires_grad=False), G.activate(G.to_params(sc, requires_grad=False))[0], cam, cfg)
        dx, dy, cb = 0.5 - float(pr["mx"][0]), 0.5 - float(pr["my"][0]), float(pr["cb"][0])
        if np.sign(dx) * np.sign(dy) == np.sign(cb) and dx != 0 and dy != 0:
            break
    else:
        raise AssertionError("no aligned offset")
    Gm, Gr, _ = _screen(sc, cam, cfg, tg, 1.0)
    assert np.all(np.abs(Gr[0]) > 0)
    # the pixel-centre offsets and the conic make both centre terms of each coordinate one sign
    assert np.allclose(Gm[0], np.abs(Gr[0]), rtol=1e-9, atol=0), (Gm[0], Gr[0])


def test_pixel_masks_partition_the_loss_and_its_gradient(tiny):
    """The loss is a sum over pixels, so restricting it to a set of pixels and to the rest
    gives two losses and two gradients that add up to the whole (linearity over a partition);
    a mask that holds everywhere changes nothing, one that holds nowhere gives exactly zero, and
    the magnitude bounds of the two halves add up to the whole's."""
    cfg = oracle.make_config()
    cam = tiny.cameras[0]
    v = oracle.prepare_view(tiny.scene, cam, cfg)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
    tg = [(img + synth.target_noise(img.shape, 0.02, tiny.seed, 0)).astype(np.float32)]
    H, W = cam.height, cam.width
    rng = np.random.default_rng(5)
    mask = np.zeros((H, W), bool)
    for ty, tx in rng.integers(0, [H // 16, W // 16], size=(12, 2)):  # whole tiles, like the device test
        mask[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = True
    L, g, _ = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, tg)
    La, ga, _ = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, tg, masks=[mask])
    Lb, gb, _ = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, tg, masks=[~mask])
    L1, g1, _ = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, tg, masks=[np.ones((H, W), bool)])
    L0, g0, _ = G.loss_and_grad(tiny.scene, tiny.cameras, cfg, tg, masks=[np.zeros((H, W), bool)])
    assert 0.0 < La < L and La + Lb == pytest.approx(L, rel=1e-12)
    assert L1 == L and L0 == 0.0
    for k in G.PARAM_KEYS:
        np.testing.assert_allclose(ga[k] + gb[k], g[k], rtol=1e-9, atol=1e-15 * np.abs(g[k]).max())
        assert np.array_equal(g1[k], g[k])
        assert not np.any(g0[k])
        assert np.count_nonzero(ga[k]) > 0
    Ma = G.loss_grad_magnitude(tiny.scene, tiny.cameras, cfg, tg, masks=[mask])
    Mb = G.loss_grad_magnitude(tiny.scene, tiny.cameras, cfg, tg, masks=[~mask])
    M = G.loss_grad_magnitude(tiny.scene, tiny.cameras, cfg, tg)
    for k in G.PARAM_KEYS:
        np.testing.assert_allclose(Ma[k] + Mb[k], M[k], rtol=1e-9, atol=1e-15 * M[k].max())
        assert np.all(np.abs(ga[k]) <= Ma[k] * (1 + 1e-9) + 1e-300)
