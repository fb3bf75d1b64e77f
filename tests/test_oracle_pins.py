"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test ties one oracle function to something independent of its own code: the
mathematical definition re-evaluated by brute force, a closed form, an invariant, or a
textbook library routine (scipy's spherical harmonics and rotations, numpy's stable sort).
"""
import math

import numpy as np
import pytest
import scipy.special as sps
from scipy.spatial.transform import Rotation

import oracle
import synth

CFG = oracle.make_config()


# ------------------------------------------------------------------------------------------
# exp2r: reproducible binary32 exp2
# ------------------------------------------------------------------------------------------

def test_exp2r_accuracy_against_exp2():
    y = np.linspace(-125.0, 125.0, 200_001, dtype=np.float32)
    got = oracle.exp2r(y).astype(np.float64)
    ref = np.exp2(y.astype(np.float64))
    rel = np.abs(got - ref) / ref
    # degree-6 Taylor remainder (ln2/2)^7/7! = 1.2e-7 plus a few binary32 roundings
    assert rel.max() < 4e-7


def test_exp2r_exact_on_integers_and_monotone():
    ints = np.arange(-125, 126, dtype=np.float32)
    assert np.array_equal(oracle.exp2r(ints), np.exp2(ints.astype(np.float64)).astype(np.float32))
    y = np.linspace(-9.0, 0.5, 400_001, dtype=np.float32)
    g = oracle.exp2r(y)
    assert np.all(np.diff(g) >= 0)


def test_exp2r_clamps_nan_and_range():
    out = oracle.exp2r(np.array([np.nan, -1e9, 1e9], np.float32))
    assert out[0] == np.float32(2.0 ** -125) and out[1] == np.float32(2.0 ** -125)
    assert out[2] == np.float32(2.0 ** 125)


# ------------------------------------------------------------------------------------------
# activation: covariance and opacity
# ------------------------------------------------------------------------------------------

def _scene(means, log_scales, quats, logits, sh=None):
    n = means.shape[1]
    if sh is None:
        sh = np.zeros((16, 3, n), np.float32)
    return synth.Scene(means.astype(np.float32), log_scales.astype(np.float32),
                       quats.astype(np.float32), logits.astype(np.float32), sh.astype(np.float32))


def test_activate_against_scipy_rotation():
    rng = np.random.default_rng(3)
    n = 500
    q = rng.normal(size=(4, n))
    ls = rng.normal(-2.0, 1.0, size=(3, n))
    sc = _scene(np.zeros((3, n)), ls, q, rng.normal(0, 2, size=n))
    cov, op = oracle.activate(sc)
    R = Rotation.from_quat(np.stack([q[1], q[2], q[3], q[0]], axis=1)).as_matrix()  # scalar last
    s2 = np.exp(2.0 * ls.T)
    ref = np.einsum("nij,nj,nkj->nik", R, s2, R)
    got = np.stack([[cov[0], cov[1], cov[2]], [cov[1], cov[3], cov[4]], [cov[2], cov[4], cov[5]]]).transpose(2, 0, 1)
    scale = s2.max(axis=1)[:, None, None]
    assert np.max(np.abs(got - ref) / scale) < 2e-6
    assert np.max(np.abs(op - sps.expit(sc.opacity_logits.astype(np.float64)))) < 2e-7


def test_activate_identity_quaternion_and_zero_logit():
    ls = np.array([[-1.0], [-2.0], [-3.0]])
    sc = _scene(np.zeros((3, 1)), ls, np.array([[2.0], [0.0], [0.0], [0.0]]), np.zeros(1))
    cov, op = oracle.activate(sc)
    np.testing.assert_allclose(cov[[0, 3, 5], 0], np.exp(2 * ls[:, 0]), rtol=1e-6)
    assert cov[1, 0] == 0 and cov[2, 0] == 0 and cov[4, 0] == 0
    assert op[0] == np.float32(0.5)


# ------------------------------------------------------------------------------------------
# projection (EWA), SH colour, tile rectangle
# ------------------------------------------------------------------------------------------

def test_sh_basis_against_scipy():
    rng = np.random.default_rng(5)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                z = sps.sph_harm_y(l, abs(m), theta, phi)  # complex, Condon-Shortley phase included
                ref = z.real if m == 0 else math.sqrt(2) * (z.real if m > 0 else z.imag)
                assert abs(Y[l * (l + 1) + m] - ref) < 1e-12, (l, m)
    # index order of the paper, (l, m) -> l(l+1)+m+1: Y_1 constant, Y_2..Y_4 = -y, z, -x (scaled)
    Y = oracle.sh_basis([0.0, 0.0, 1.0])
    assert abs(Y[0] - 0.5 / math.sqrt(math.pi)) < 1e-15 and abs(Y[2] - math.sqrt(3 / (4 * math.pi))) < 1e-15


def test_axis_aligned_splat_on_optical_axis():
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 128, 96)
    sigma = 0.05
    sc = _scene(np.zeros((3, 1)), np.full((3, 1), math.log(sigma)), np.array([[1.0], [0], [0], [0]]), np.zeros(1))
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    f = cam.fy
    expect = f * f * sigma * sigma / 9.0 + 0.3
    assert pr["cov2d"][0, 0] == pytest.approx(expect, rel=2e-6)
    assert pr["cov2d"][2, 0] == pytest.approx(expect, rel=2e-6)
    assert abs(pr["cov2d"][1, 0]) < 1e-6 * expect
    assert pr["mean2d"][0, 0] == pytest.approx(64.0, abs=1e-5) and pr["mean2d"][1, 0] == pytest.approx(48.0, abs=1e-5)
    assert pr["conic"][0, 0] == pytest.approx(1.0 / expect, rel=4e-6)
    assert pr["radius"][0] == math.ceil(3.0 * math.sqrt(expect) - 1e-6) or pr["radius"][0] == math.ceil(3 * math.sqrt(expect))
    assert pr["depth"][0] == np.float32(3.0)


def _numeric_jacobian(cam, p):
    """d(pixel)/d(world point) by central differences of the pinhole map (binary64)."""
    R = cam.w2c.reshape(3, 4)[:, :3].astype(np.float64)
    t = cam.w2c.reshape(3, 4)[:, 3].astype(np.float64)

    def proj(x):
        c = R @ x + t
        return np.array([cam.fx * c[0] / c[2] + cam.cx, cam.fy * c[1] / c[2] + cam.cy])

    J = np.zeros((2, 3))
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        J[:, j] = (proj(p + e) - proj(p - e)) / (2 * h)
    return proj(p), J


def test_projection_is_linearised_pinhole(tiny):
    sc, cam = tiny.scene, tiny.cameras[0]
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    vis = np.nonzero(pr["touched"])[0]
    assert vis.size > 500
    checked = 0
    for k in vis[:300]:
        mu = sc.means[:, k].astype(np.float64)
        m2, J = _numeric_jacobian(cam, mu)
        # only splats inside the Jacobian clamp region follow the plain linearisation
        c = cam.w2c.reshape(3, 4)[:, :3] @ mu + cam.w2c.reshape(3, 4)[:, 3]
        if abs(c[0] / c[2]) > 1.3 * 0.5 * cam.width / cam.fx or abs(c[1] / c[2]) > 1.3 * 0.5 * cam.height / cam.fy:
            continue
        S = np.array([[cov[0, k], cov[1, k], cov[2, k]], [cov[1, k], cov[3, k], cov[4, k]], [cov[2, k], cov[4, k], cov[5, k]]], np.float64)
        ref = J @ S @ J.T + 0.3 * np.eye(2)
        got = np.array([[pr["cov2d"][0, k], pr["cov2d"][1, k]], [pr["cov2d"][1, k], pr["cov2d"][2, k]]])
        assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref)) + 1e-6
        assert np.max(np.abs(pr["mean2d"][:, k] - m2)) < 1e-4
        checked += 1
    assert checked > 200


def test_colour_dc_only():
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 64, 64)
    sh = np.zeros((16, 3, 1), np.float32)
    sh[0, :, 0] = [1.0, -0.2, -3.0]
    sc = _scene(np.zeros((3, 1)), np.full((3, 1), -3.0), np.array([[1.0], [0], [0], [0]]), np.zeros(1), sh)
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    y0 = 0.5 / math.sqrt(math.pi)
    np.testing.assert_allclose(pr["rgb"][:, 0], [max(0, v * y0 + 0.5) for v in sh[0, :, 0].astype(np.float64)], rtol=1e-12)


@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_rect_encloses_square_and_clamps(tiny, tile):
    """The tile rectangle is every tile of the view that meets the square of half-side r around the
    centre, by enumeration, for the three tile shapes (width and height used on their own axes)."""
    sc, cam = tiny.scene, tiny.cameras[0]
    tw, th = tile
    cfg = oracle.make_config(tile_w=tw, tile_h=th)
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, cfg, op)
    tx, ty = oracle.tiles_of(cam, cfg)
    for k in np.nonzero(pr["touched"])[0][:400]:
        mx, my, r = pr["mean2d"][0, k], pr["mean2d"][1, k], pr["radius"][k]
        want = [(x, y) for y in range(ty) for x in range(tx)
                if x * tw <= mx + r and (x + 1) * tw > mx - r and y * th <= my + r and (y + 1) * th > my - r]
        x0, y0, x1, y1 = pr["rect"][:, k]
        got = [(x, y) for y in range(y0, y1) for x in range(x0, x1)]
        assert sorted(got) == sorted(want)
        kept = [t for t in got if len(got) > oracle.CULL_MAX_TILES or oracle.tile_hit(pr, k, t[0], t[1], cfg)]
        assert pr["touched"][k] == len(kept)


def test_cull_behind_and_near():
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 64, 64)
    means = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [-3.5, -2.9, 0.0]])  # behind, inside near, visible
    sc = _scene(means, np.full((3, 3), -3.0), np.tile([[1.0], [0], [0], [0]], (1, 3)), np.zeros(3))
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    assert list(pr["touched"][:2]) == [0, 0] and pr["touched"][2] > 0


def test_near_plane_is_exclusive():
    """A splat is culled when its camera-space z <= near_z: exactly on the plane it goes, one
    binary32 step beyond it stays (identity world-to-camera map, so z is the stored mean)."""
    near = np.float32(CFG.near_z)
    cam = synth.Camera(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32), 40.0, 40.0, 32.0, 32.0, 64, 64)
    zs = [near, np.nextafter(near, np.float32(1.0))]
    means = np.array([[0.0, 0.0], [0.0, 0.0], zs], np.float32)
    sc = _scene(means, np.full((3, 2), -3.0), np.tile([[1.0], [0], [0], [0]], (1, 2)), np.zeros(2))
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    assert pr["touched"][0] == 0 and pr["touched"][1] > 0


def test_cull_limit_is_64_tiles():
    """A needle-shaped splat along the image diagonal: with a rectangle of 33 to 64 tiles its
    off-diagonal corner tiles are dropped by the tile test; with more than 64 tiles every tile is
    kept."""
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 256, 256)
    c, s_ = math.cos(math.pi / 8), math.sin(math.pi / 8)  # 45 degrees about z
    means = np.zeros((3, 2))
    log_scales = np.array([[math.log(0.226), math.log(0.4)], [math.log(0.02)] * 2, [math.log(0.02)] * 2])
    quats = np.array([[c, c], [0, 0], [0, 0], [s_, s_]])
    sc = _scene(means, log_scales, quats, np.full(2, 3.0))
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    x0, y0, x1, y1 = pr["rect"]
    area = (x1 - x0) * (y1 - y0)
    assert 32 < area[0] <= oracle.CULL_MAX_TILES and 0 < pr["touched"][0] < area[0]
    assert area[1] > oracle.CULL_MAX_TILES and pr["touched"][1] == area[1]


# ------------------------------------------------------------------------------------------
# binning and sort
# ------------------------------------------------------------------------------------------

def test_bin_sort_against_numpy_stable_sort(tiny):
    _check_bin_sort(tiny.scene, tiny.cameras[0])


def test_bin_sort_keeps_emission_order_for_equal_keys(tiny):
    """Splat 2j + 1 a copy of splat 2j's position (its own shape and opacity): the pair has the
    same depth, so wherever both touch a tile their keys are equal and a stable sort keeps them in
    emission order (k ascending)."""
    sc = tiny.scene
    means = sc.means.copy()
    means[:, 1::2] = means[:, 0:means.shape[1] - 1:2]
    dup = synth.Scene(means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh)
    ties = _check_bin_sort(dup, tiny.cameras[0])
    assert ties > 100


def test_bin_sort_with_frame_bases(tiny):
    """A view inside a multi-view frame: with tile base B and value base V its keys carry global
    tiles t + B, its values are V + k, and its ranges (indexed by the view's own tiles), order and
    emission indices are those of the view alone."""
    sc, cam = tiny.scene, tiny.cameras[0]
    v = oracle.prepare_view(sc, cam, CFG)
    B, V = 123_457, 3 * sc.n
    keys, vals, emit, ranges = oracle.bin_sort(v, cam, CFG, tile_base=B, val_base=V)
    assert v["keys"].size > 1000
    assert np.array_equal(keys >> np.uint64(32), (v["keys"] >> np.uint64(32)) + np.uint64(B))
    assert np.array_equal(keys & np.uint64(0xFFFFFFFF), v["keys"] & np.uint64(0xFFFFFFFF))
    assert np.array_equal(vals, v["vals"] + np.uint32(V))
    assert np.array_equal(emit, v["emit"]) and np.array_equal(ranges, v["ranges"])


def _check_bin_sort(sc, cam):
    """The oracle's keys, values, emission indices and tile ranges against numpy's stable argsort
    of keys emitted by enumeration, for the three tile shapes; returns the number of equal
    adjacent keys seen."""
    ties = 0
    for tw, th in [(16, 16), (8, 32), (32, 8)]:
        cfg = oracle.make_config(tile_w=tw, tile_h=th)
        v = oracle.prepare_view(sc, cam, cfg)
        tx, ty = oracle.tiles_of(cam, cfg)
        keys, vals = [], []
        for k in range(sc.n):
            x0, y0, x1, y1 = v["rect"][:, k]
            dbits = int(np.float32(v["depth"][k]).view(np.uint32))
            big = (x1 - x0) * (y1 - y0) > oracle.CULL_MAX_TILES
            for y in range(y0, y1):
                for x in range(x0, x1):
                    if big or oracle.tile_hit(v, k, x, y, cfg):
                        keys.append(((y * tx + x) << 32) | dbits)
                        vals.append(k)
        keys = np.array(keys, np.uint64)
        order = np.argsort(keys, kind="stable")
        ties += int(np.count_nonzero(np.diff(keys[order].astype(np.int64)) == 0))
        assert np.array_equal(v["keys"], keys[order])
        assert np.array_equal(v["vals"], np.array(vals, np.uint32)[order])
        assert np.array_equal(v["emit"], order.astype(np.uint32))
        tiles = (keys[order] >> np.uint64(32)).astype(np.int64)
        for t in range(tx * ty):
            idx = np.nonzero(tiles == t)[0]
            if idx.size:
                assert tuple(v["ranges"][t]) == (idx[0], idx[-1] + 1)
            else:
                assert v["ranges"][t][0] == v["ranges"][t][1]
    return ties


def _random_splats(rng, m, tile):
    """Splats around one tile: centres within 1.5 tiles of it, 2D covariances of every
    orientation and anisotropy (low-pass 0.3 added), opacities from 0.004 to 0.99."""
    out = []
    for _ in range(m):
        mx = float(rng.uniform(-1.5, 2.5) * tile[0])
        my = float(rng.uniform(-1.5, 2.5) * tile[1])
        th = rng.uniform(0, np.pi)
        s1, s2 = np.exp(rng.uniform(np.log(0.3), np.log(12.0), 2))
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        S = R @ np.diag([s1 * s1, s2 * s2]) @ R.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        kA = -0.5 * math.log2(math.e)
        A, B, C = np.float32(Q[0, 0] * kA), np.float32(-Q[0, 1] * math.log2(math.e)), np.float32(Q[1, 1] * kA)
        o = float(np.exp(rng.uniform(np.log(0.004), np.log(0.99))))
        out.append((np.float32(mx), np.float32(my), A, B, C, np.float32(o)))
    return out


def _tile_alpha_max(sp, tile, step):
    """Largest o 2^p over a lattice of the tile's pixel-centre rectangle (binary64)."""
    mx, my, A, B, C, o = (float(x) for x in sp)
    xs = np.arange(0.5, tile[0] - 0.5 + 1e-9, step)
    ys = np.arange(0.5, tile[1] - 0.5 + 1e-9, step)
    u = xs[None, :] - mx
    v = ys[:, None] - my
    p = A * u * u + B * u * v + C * v * v
    return o * np.exp2(p.max())


def test_tile_test_is_conservative_and_tight():
    """Brute force over pixel centres: a tile that some pixel centre gives alpha >= alpha_min
    is always kept; a kept tile comes within the test's margin of alpha_min somewhere on its
    pixel-centre rectangle (sampled at 1/8 pixel, edges included)."""
    rng = np.random.default_rng(11)
    amin = float(CFG.alpha_min)
    kept = dropped = near = 0
    for tw, th in [(16, 16), (8, 32), (32, 8)]:
        cfg = oracle.make_config(tile_w=tw, tile_h=th)
        for sp in _random_splats(rng, 700, (tw, th)):
            proj = dict(mean2d=np.array([[sp[0]], [sp[1]]], np.float32),
                        qcoef=np.array([[sp[2]], [sp[3]], [sp[4]]], np.float32), opacity=np.array([sp[5]], np.float32))
            hit = oracle.tile_hit(proj, 0, 0, 0, cfg)
            on_pixels = _tile_alpha_max(sp, (tw, th), 1.0)
            if on_pixels >= amin * (1 + 1e-6):
                assert hit, sp
            dense = _tile_alpha_max(sp, (tw, th), 0.125)
            if hit:
                kept += 1
                assert dense >= amin * 2.0 ** -0.25, sp
                near += dense < amin
            else:
                dropped += 1
                assert dense < amin * 1.001, sp
    assert kept > 300 and dropped > 300 and near < 0.03 * kept
    # on the boundary: opacity set so that the sampled maximum is alpha_min x f
    both = 0
    for sp in _random_splats(rng, 1500, (16, 16)):
        peak = _tile_alpha_max(sp, (16, 16), 0.125) / float(sp[5])
        if not 1e-30 < peak:
            continue
        res = []
        for f in (1.002, 0.95):
            o = np.float32(amin * f / peak)
            if not 0.0 < o < 1.0:
                break
            proj = dict(mean2d=np.array([[sp[0]], [sp[1]]], np.float32),
                        qcoef=np.array([[sp[2]], [sp[3]], [sp[4]]], np.float32), opacity=np.array([o], np.float32))
            res.append(oracle.tile_hit(proj, 0, 0, 0, CFG))
        if len(res) == 2:
            assert res[0]  # the continuous maximum passes alpha_min: kept
            both += 1
            dropped += not res[1]
            near += res[1]
    # the margin keeps only a sliver of tiles whose maximum is 5 % short of alpha_min
    assert both > 300 and near < 0.05 * both
    # a splat centred on a pixel centre (exponent 0 there): 3e-5 short of alpha_min is inside the
    # margin (kept), 1 % short is not (dropped)
    for f, want in ((1.0 - 3e-5, True), (0.99, False)):
        proj = dict(mean2d=np.array([[7.5], [7.5]], np.float32),
                    qcoef=np.array([[-0.05], [0.0], [-0.05]], np.float32),
                    opacity=np.array([np.float32(amin * f)], np.float32))
        assert oracle.tile_hit(proj, 0, 0, 0, CFG) == want, f


def test_tile_test_agrees_with_rendered_alphas(tiny):
    """Every (pixel, splat) pair the compositor takes lies in a kept tile, and nearly every
    kept instance of the tiny view has a pixel whose alpha (in binary64) reaches alpha_min."""
    sc, cam = tiny.scene, tiny.cameras[0]
    v = oracle.prepare_view(sc, cam, CFG)
    pix, ks, pos = oracle.pixel_lists(v, v["vals"], v["ranges"], cam, CFG)
    tx, _ = oracle.tiles_of(cam, CFG)
    tile_of_pix = (pix // cam.width // 16) * tx + (pix % cam.width) // 16
    kept = set(zip((v["keys"] >> np.uint64(32)).astype(np.int64).tolist(), v["vals"].astype(np.int64).tolist()))
    assert all((int(t), int(k)) in kept for t, k in zip(tile_of_pix, ks))
    hit = 0
    for t, k in list(kept)[:3000]:
        x, y = t % tx, t // tx
        sp = (v["mean2d"][0, k] - 16 * x, v["mean2d"][1, k] - 16 * y, *v["qcoef"][:, k], v["opacity"][k])
        hit += _tile_alpha_max(sp, (16, 16), 1.0) >= CFG.alpha_min * 0.99
    assert hit >= 0.97 * min(3000, len(kept))


def _full_rect_lists(v, cam, cfg):
    """Whole-rectangle binning written out with numpy: per tile, every splat whose 3-sigma
    rectangle covers it, stably ordered by depth bits."""
    tx, ty = oracle.tiles_of(cam, cfg)
    keys, vals = [], []
    for k in np.nonzero(v["rect"][2] > v["rect"][0])[0]:
        x0, y0, x1, y1 = v["rect"][:, k]
        d = int(np.float32(v["depth"][k]).view(np.uint32))
        for y in range(y0, y1):
            for x in range(x0, x1):
                keys.append(((y * tx + x) << 32) | d)
                vals.append(k)
    keys = np.array(keys, np.uint64)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], np.array(vals, np.uint32)[order]
    t = (keys >> np.uint64(32)).astype(np.int64)
    ranges = np.zeros((tx * ty, 2), np.uint32)
    ranges[:, 0] = np.searchsorted(t, np.arange(tx * ty), "left")
    ranges[:, 1] = np.searchsorted(t, np.arange(tx * ty), "right")
    return vals, ranges


def test_culled_binning_renders_and_removes_like_whole_rectangles(tiny):
    """Images, transmittances and per-splat removal effects from the culled lists equal those
    from whole-rectangle lists bit for bit: culling only drops pairs the compositor skips."""
    sc, cam = tiny.scene, tiny.cameras[0]
    v = oracle.prepare_view(sc, cam, CFG)
    fv, fr = _full_rect_lists(v, cam, CFG)
    assert fv.size > v["vals"].size * 1.2
    a = oracle.render(v, v["vals"], v["ranges"], cam, CFG)
    b = oracle.render(v, fv, fr, cam, CFG)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    tgt = (a[0] + synth.target_noise(a[0].shape, 0.02, 5, 0)).astype(np.float32)
    da, ia = oracle.removal_effect(v, v["vals"], v["ranges"], cam, CFG, tgt)
    db, ib = oracle.removal_effect(v, fv, fr, cam, CFG, tgt)
    assert np.array_equal(da, db) and np.array_equal(ia, ib)
    assert np.count_nonzero(da) > 500


def test_whole_rectangle_binning_against_numpy_enumeration(tiny):
    """The oracle's binning with the tile test switched off (whole_rect) equals the numpy
    enumeration of every 3-sigma rectangle tile stably sorted by (tile, depth bits), for the
    three tile shapes; it holds the culled binning's lists as order-preserving subsequences."""
    sc, cam = tiny.scene, tiny.cameras[0]
    for tw, th in [(16, 16), (8, 32), (32, 8)]:
        cfg = oracle.make_config(tile_w=tw, tile_h=th)
        v = oracle.prepare_view(sc, cam, cfg)
        keys, vals, emit, ranges = oracle.bin_sort(v, cam, cfg, whole_rect=True)
        fv, fr = _full_rect_lists(v, cam, cfg)
        assert np.array_equal(vals, fv)
        empty = fr[:, 1] == fr[:, 0]  # the oracle writes (0, 0) for an empty tile
        assert np.array_equal(ranges[~empty], fr[~empty]) and np.all(ranges[empty] == 0)
        assert vals.size > 1.2 * v["vals"].size
        for t in range(ranges.shape[0]):
            whole = list(vals[ranges[t, 0]:ranges[t, 1]])
            culled = list(v["vals"][v["ranges"][t, 0]:v["ranges"][t, 1]])
            it = iter(whole)
            assert all(k in it for k in culled)  # subsequence test: consumes `it` in order


def test_depth_bits_order_matches_numeric_order():
    d = np.sort(np.random.default_rng(1).uniform(0.2, 1e4, 100_000).astype(np.float32))
    assert np.all(np.diff(d.view(np.uint32).astype(np.int64)) >= 0)


# ------------------------------------------------------------------------------------------
# compositing and removal effect on hand-built splats (closed forms)
# ------------------------------------------------------------------------------------------

def test_jacobian_clamp_freezes_the_footprint_beyond_the_limit():
    """The Jacobian is taken at the camera-space point with x / z clamped to 1.3 times the half
    field of view: an isotropic splat at a fixed depth has one 2D covariance for every position
    beyond that limit, and a smaller one inside it (the footprint of the plain linearisation grows
    with (x / z)^2)."""
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 128, 96)
    W = cam.w2c.reshape(3, 4).astype(np.float64)
    lim = 1.3 * 0.5 * cam.width / cam.fx
    z = 3.0
    ratios = [0.5 * lim, 1.5 * lim, 2.0 * lim, 3.0 * lim]
    cam_pts = np.array([[r * z, 0.0, z] for r in ratios])
    world = (W[:, :3].T @ (cam_pts.T - W[:, 3:4]))  # x_c = R x + t  ->  x = R^T (x_c - t)
    n = len(ratios)
    sc = _scene(world, np.full((3, n), math.log(3.0)), np.tile([[1.0], [0], [0], [0]], n), np.full(n, 4.0))
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    assert np.all(pr["touched"] > 0)
    c2 = pr["cov2d"].astype(np.float64)
    for j in (2, 3):
        np.testing.assert_allclose(c2[:, j], c2[:, 1], rtol=1e-5, atol=1e-3)
    assert c2[0, 0] < 0.9 * c2[0, 1]


def test_projection_with_unequal_focal_lengths():
    """A camera with fx = 1.6 fy and an off-centre principal point: centres and 2D covariances
    still follow the finite-difference linearisation of its pinhole map (fx on x, fy on y)."""
    sc = synth.uniform_cube_scene(400, 17)
    base = synth.look_at_camera((0.3, -0.2, -3.0), 160, 90)
    cam = synth.Camera(base.w2c, 1.6 * base.fy, base.fy, 0.45 * base.width, 0.55 * base.height, base.width,
                       base.height)
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    W = cam.w2c.reshape(3, 4).astype(np.float64)
    checked = 0
    for k in np.nonzero(pr["touched"])[0]:
        mu = sc.means[:, k].astype(np.float64)
        c = W[:, :3] @ mu + W[:, 3]
        if abs(c[0] / c[2]) > 1.3 * 0.5 * cam.width / cam.fx or abs(c[1] / c[2]) > 1.3 * 0.5 * cam.height / cam.fy:
            continue
        m2, J = _numeric_jacobian(cam, mu)
        S = np.array([[cov[0, k], cov[1, k], cov[2, k]], [cov[1, k], cov[3, k], cov[4, k]],
                      [cov[2, k], cov[4, k], cov[5, k]]], np.float64)
        ref = J @ S @ J.T + 0.3 * np.eye(2)
        got = np.array([[pr["cov2d"][0, k], pr["cov2d"][1, k]], [pr["cov2d"][1, k], pr["cov2d"][2, k]]])
        assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref)) + 1e-6
        assert np.max(np.abs(pr["mean2d"][:, k] - m2)) < 1e-4
        checked += 1
    assert checked > 100


def _flat_view(opac, rgb, depth, w=16, h=16):
    """Splats whose exponent is 0 everywhere (alpha = opacity exactly), all in one tile."""
    n = len(opac)
    v = dict(
        mean2d=np.zeros((2, n), np.float32), qcoef=np.zeros((3, n), np.float32),
        opacity=np.array(opac, np.float32), rgb=np.ascontiguousarray(np.array(rgb, np.float64).T),
        depth=np.array(depth, np.float32),
    )
    order = np.argsort(np.array(depth, np.float32), kind="stable")
    vals = order.astype(np.uint32)
    ranges = np.array([[0, n]], np.uint32)
    cam = synth.Camera(np.zeros(12, np.float32), 1.0, 1.0, 0.0, 0.0, w, h)
    return v, vals, ranges, cam


def test_one_splat_closed_form():
    c0 = np.array([0.7, 0.2, 0.4])
    v, vals, ranges, cam = _flat_view([0.6], [c0], [1.0])
    cfg = oracle.make_config(t_min=0.0)
    img, t32, t64, nl = oracle.render(v, vals, ranges, cam, cfg)
    a = float(np.float32(0.6))
    np.testing.assert_allclose(img[:, 0, 0], a * c0, rtol=1e-15)
    assert t64[0, 0] == pytest.approx(1 - a, rel=1e-15) and nl[0, 0] == 1
    ct = np.array([0.1, 0.5, 0.3], np.float32)
    tgt = np.broadcast_to(ct[:, None, None], (3, 16, 16))
    d, imp = oracle.removal_effect(v, vals, ranges, cam, cfg, tgt)
    C0 = a * c0
    per_pix = np.sum(C0 * (C0 - 2 * (C0 - ct.astype(np.float64))))  # PD = -alpha c0
    assert d[0] == pytest.approx(256 * per_pix, rel=1e-12)
    assert imp[0] == pytest.approx(256 * a, rel=1e-12)


def test_two_splat_closed_form_front_and_back():
    c0, c1 = np.array([0.9, 0.1, 0.3]), np.array([0.2, 0.8, 0.5])
    v, vals, ranges, cam = _flat_view([0.99, 0.7], [c0, c1], [1.0, 2.0])
    cfg = oracle.make_config(t_min=0.0, alpha_max=0.99)
    a0, a1 = float(np.float32(0.99)), float(np.float32(0.7))
    img, *_ = oracle.render(v, vals, ranges, cam, cfg)
    C = a0 * c0 + (1 - a0) * a1 * c1
    np.testing.assert_allclose(img[:, 3, 5], C, rtol=1e-14)
    tgt = np.zeros((3, 16, 16), np.float32)
    d, imp = oracle.removal_effect(v, vals, ranges, cam, cfg, tgt)
    pd_front = a0 * (a1 * c1 - c0)
    pd_back = -(1 - a0) * a1 * c1  # the 1/(1 - alpha) renormalisation at alpha_0 = 0.99
    dse = lambda pd: np.sum(pd * pd + 2 * pd * C)
    assert d[0] == pytest.approx(256 * dse(pd_front), rel=1e-11)
    assert d[1] == pytest.approx(256 * dse(pd_back), rel=1e-9)
    assert imp[0] == pytest.approx(256 * a0, rel=1e-12) and imp[1] == pytest.approx(256 * (1 - a0) * a1, rel=1e-9)


def test_alpha_clamp_and_threshold_and_termination():
    # opacity above alpha_max is clamped; below alpha_min never composites; T_min stops
    v, vals, ranges, cam = _flat_view([1.0, 0.003, 0.5], [[1, 1, 1], [1, 0, 0], [0, 1, 0]], [1.0, 2.0, 3.0])
    cfg = oracle.make_config(t_min=0.0)
    img, t32, t64, nl = oracle.render(v, vals, ranges, cam, cfg)
    a0 = float(np.float32(0.99))
    a2 = float(np.float32(0.5))
    np.testing.assert_allclose(img[:, 0, 0], a0 * np.ones(3) + (1 - a0) * a2 * np.array([0, 1, 0]), rtol=1e-14)
    assert nl[0, 0] == 3
    cfg2 = oracle.make_config(t_min=0.006)
    img2, t32b, _, nl2 = oracle.render(v, vals, ranges, cam, cfg2)
    assert nl2[0, 0] == 1 and t32b[0, 0] == np.float32(1.0) - np.float32(0.99)  # stops before the last splat


def test_termination_ends_the_pixel():
    """T_min ends the walk at the first splat that would take T below it: 0.99 then 0.98 leave
    T = 2e-4; 0.9 would leave 2e-5 < 1e-4, so the pixel stops there, and a fainter splat after it
    (0.1, which would leave 1.8e-4) is not composited either."""
    v, vals, ranges, cam = _flat_view([0.99, 0.98, 0.9, 0.1], [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]],
                                      [1.0, 2.0, 3.0, 4.0])
    img, t32, t64, nl = oracle.render(v, vals, ranges, cam, oracle.make_config(t_min=1e-4))
    a0, a1 = float(np.float32(0.99)), float(np.float32(0.98))
    np.testing.assert_allclose(img[:, 0, 0], [a0, (1 - a0) * a1, 0.0], rtol=1e-14, atol=0)
    assert nl[0, 0] == 2 and t32[0, 0] >= np.float32(1e-4)
    tgt = np.zeros(img.shape, np.float32)
    d, imp = oracle.removal_effect(v, vals, ranges, cam, oracle.make_config(t_min=1e-4), tgt)
    assert d[2] == 0.0 and d[3] == 0.0 and imp[2] == 0.0 and imp[3] == 0.0


# ------------------------------------------------------------------------------------------
# tiny scene: definition, invariants
# ------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny_view(tiny):
    sc, cam = tiny.scene, tiny.cameras[0]
    v = oracle.prepare_view(sc, cam, CFG)
    img, t32, t64, nl = oracle.render(v, v["vals"], v["ranges"], cam, CFG)
    tgt = (img + synth.target_noise(img.shape, 0.02, tiny.seed, 0)).astype(np.float32)
    return v, img, t32, t64, nl, tgt


def test_removal_effect_equals_definition_bruteforce(tiny, tiny_view):
    v, img, t32, t64, nl, tgt = tiny_view
    cam = tiny.cameras[0]
    cfg0 = oracle.make_config(t_min=0.0)
    img0, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg0)
    d, _ = oracle.removal_effect(v, v["vals"], v["ranges"], cam, cfg0, tgt)
    nz = 0
    for k in range(100):
        b = oracle.removal_bruteforce(v, v["vals"], v["ranges"], cam, cfg0, tgt, img0, k)
        assert abs(d[k] - b) <= 1e-10 * abs(b) + 1e-13, k
        nz += b != 0
    assert nz > 50


def test_dmse_is_the_change_in_mean_squared_error(tiny):
    """dMSE_k is the change, when splat k alone is removed, of the mean squared error averaged over
    the views (np.mean over each view's 3 x H x W values, then over views; two views of different
    sizes; T_min = 0 so that the removal is exact), and the importances add up to the mean
    coverage 1 - T_final averaged the same way."""
    sc = tiny.scene
    cams = [tiny.cameras[0], synth.look_at_camera((1.5, 0.4, -2.6), 96, 64)]
    cfg0 = oracle.make_config(t_min=0.0)
    tgts, imgs, cover = [], [], []
    for v, cam in enumerate(cams):
        pv = oracle.prepare_view(sc, cam, cfg0)
        img, t32, t64, nl = oracle.render(pv, pv["vals"], pv["ranges"], cam, cfg0)
        tgts.append((img + synth.target_noise(img.shape, 0.02, 7, v)).astype(np.float32))
        imgs.append(img)
        cover.append(np.mean(1.0 - t64))
    d, imp = oracle.dmse(sc, cams, cfg0, tgts)
    assert imp.sum() == pytest.approx(np.mean(cover), rel=1e-12)
    checked = 0
    for k in np.argsort(-np.abs(d))[:12]:
        keep = np.ones(sc.n, bool)
        keep[k] = False
        sub = sc.subset(keep)
        change = []
        for cam, img, tgt in zip(cams, imgs, tgts):
            pv = oracle.prepare_view(sub, cam, cfg0)
            img_k, *_ = oracle.render(pv, pv["vals"], pv["ranges"], cam, cfg0)
            t = tgt.astype(np.float64)
            change.append(np.mean((img_k - t) ** 2) - np.mean((img - t) ** 2))
        assert d[k] == pytest.approx(np.mean(change), rel=1e-9, abs=1e-15), k
        checked += 1
    assert checked == 12 and np.abs(d).max() > 0


def test_per_instance_partials_add_up_per_splat(tiny, tiny_view):
    """The per-(tile, splat) partials sit at the splat's own list position: adding them up over
    each splat's instances (through the sorted values) gives its dSSE and its importance sum."""
    v, img, t32, t64, nl, tgt = tiny_view
    cam = tiny.cameras[0]
    d, imp, idse, iimp = oracle.removal_effect(v, v["vals"], v["ranges"], cam, CFG, tgt, per_instance=True)
    n = tiny.scene.n
    by_splat_d = np.zeros(n)
    by_splat_i = np.zeros(n)
    np.add.at(by_splat_d, v["vals"].astype(np.int64), idse)
    np.add.at(by_splat_i, v["vals"].astype(np.int64), iimp)
    assert np.count_nonzero(d) > 100
    np.testing.assert_allclose(by_splat_d, d, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(by_splat_i, imp, rtol=1e-9, atol=1e-12)


def test_removal_effect_pd_squared_when_target_is_render(tiny, tiny_view):
    v, img, t32, t64, nl, tgt = tiny_view
    d, _ = oracle.removal_effect(v, v["vals"], v["ranges"], tiny.cameras[0], CFG, img.astype(np.float32))
    # target = render up to binary32 rounding of the target: dSE = PD^2 + O(1e-8 PD)
    assert d.min() > -1e-6


def test_importance_sums_to_coverage(tiny, tiny_view):
    v, img, t32, t64, nl, tgt = tiny_view
    _, imp = oracle.removal_effect(v, v["vals"], v["ranges"], tiny.cameras[0], CFG, tgt)
    assert imp.sum() == pytest.approx((1.0 - t64).sum(), rel=1e-12)
    assert np.all(img >= 0)
    assert np.all(t32 >= CFG.t_min) and np.all(t32 <= 1)


def test_transparent_and_offscreen_splats_have_zero_effect(tiny):
    sc = tiny.scene
    sc2 = synth.Scene(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity_logits.copy(), sc.sh.copy())
    sc2.opacity_logits[:10] = -30.0  # alpha < alpha_min everywhere
    sc2.means[:, 10:20] = [[50.0], [50.0], [50.0]]  # far outside the view
    cam = tiny.cameras[0]
    v = oracle.prepare_view(sc2, cam, CFG)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, CFG)
    tgt = (img + 0.05).astype(np.float32)
    d, imp = oracle.removal_effect(v, v["vals"], v["ranges"], cam, CFG, tgt)
    assert np.all(d[:20] == 0.0) and np.all(imp[:20] == 0.0)
    assert np.count_nonzero(d[20:]) > 500


def test_affine_in_alpha_identity(tiny, tiny_view):
    """c is affine in each alpha_i: PD_i = c(alpha_i = 0) - c = 2 c(alpha_i/2) - 2 c(alpha_i),
    checked for whole splats by halving the opacity (alpha_min = 0, no clamp active)."""
    v, *_ = tiny_view
    cam = tiny.cameras[0]
    cfg = oracle.make_config(t_min=0.0, alpha_min=0.0, alpha_max=1.0)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, cfg)
    tgt = np.zeros_like(img, dtype=np.float32)
    for k in range(5):
        v2 = dict(v)
        v2["opacity"] = v["opacity"].copy()
        v2["opacity"][k] = v["opacity"][k] * np.float32(0.5)  # exact halving in binary32
        img_half, *_ = oracle.render(v2, v["vals"], v["ranges"], cam, cfg)
        # exp2r is the same on both renders, so alpha halves exactly except for o*G rounding
        pd_img = 2 * img_half - 2 * img  # c(alpha=0) - c(alpha)
        want = np.sum(pd_img * pd_img + 2 * pd_img * img)
        d, _ = oracle.removal_effect(v, v["vals"], v["ranges"], cam, cfg, tgt)
        assert d[k] == pytest.approx(want, rel=1e-5, abs=1e-9)


def test_dmse_view_normalisation_invariant(tiny):
    sc, cam = tiny.scene, tiny.cameras[0]
    v = oracle.prepare_view(sc, cam, CFG)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, CFG)
    tgt = (img + 0.01).astype(np.float32)
    one, i1 = oracle.dmse(sc, [cam], CFG, [tgt])
    two, i2 = oracle.dmse(sc, [cam, cam], CFG, [tgt, tgt])  # a repeated view leaves the mean unchanged
    np.testing.assert_allclose(two, one, rtol=1e-14, atol=0)
    np.testing.assert_allclose(i2, i1, rtol=1e-14)
    d, _ = oracle.removal_effect(v, v["vals"], v["ranges"], cam, CFG, tgt)
    np.testing.assert_allclose(one, d / (3 * cam.pixels), rtol=1e-14)


def test_colour_direction_is_camera_to_splat():
    # camera at (0, 0, -3), splat at (1, 0, 0): direction (1, 0, 3)/sqrt(10); only Y_2 = Y_1^0 (l=1, m=0) set
    cam = synth.look_at_camera((0.0, 0.0, -3.0), 256, 256)
    sh = np.zeros((16, 3, 1), np.float32)
    sh[2, :, 0] = 1.0
    sh[3, 1, 0] = 1.0  # green also gets Y_1^1 = -c x
    sc = _scene(np.array([[1.0], [0.0], [0.0]]), np.full((3, 1), -3.0), np.array([[1.0], [0], [0], [0]]), np.zeros(1), sh)
    cov, op = oracle.activate(sc)
    pr = oracle.project(sc, cov, cam, CFG, op)
    c1 = math.sqrt(3 / (4 * math.pi))
    d = np.array([1.0, 0.0, 3.0]) / math.sqrt(10.0)
    assert pr["touched"][0] > 0
    assert pr["rgb"][0, 0] == pytest.approx(c1 * d[2] + 0.5, rel=1e-6)
    assert pr["rgb"][1, 0] == pytest.approx(c1 * d[2] - c1 * d[0] + 0.5, rel=1e-6)


def test_threads_over_tiles_change_no_bit(tiny):
    """The oracle's render and removal effect on 1, 3 and 8 threads over tiles: images,
    transmittances, n_last, per-splat and per-instance sums identical bit for bit (every output
    has one owning tile; per-splat sums are formed from per-instance sums in tile order)."""
    sc = synth.uniform_cube_scene(5000, 77)
    cam = synth.look_at_camera((0.0, 0.3, -3.0), 200, 150)
    v = oracle.prepare_view(sc, cam, CFG)
    tgt = np.full((3, 150, 200), 0.3, np.float32)
    outs = []
    try:
        for nt in (1, 3, 8):
            oracle.set_threads(nt)
            assert oracle.get_threads() == nt
            r = oracle.render(v, v["vals"], v["ranges"], cam, CFG)
            d = oracle.removal_effect(v, v["vals"], v["ranges"], cam, CFG, tgt, per_instance=True)
            outs.append(list(r) + list(d))
    finally:
        oracle.set_threads(1)
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
    assert np.count_nonzero(outs[0][4]) > 1000


def test_removal_magnitude_bounds_the_removal_effect(tiny):
    """The rounding scale of the removal effect (oracle.removal_magnitude, a tolerance quantity):
    at least |dSSE_k| for every splat, its per-instance sums add up to the per-splat ones, and for
    one splat against a zero target (PD = -alpha c, dSE = -(alpha c)^2 per channel) it is exactly
    four times |dSSE| (|T alpha c| (2 |PD| + 2 |c|) = 4 (alpha c)^2)."""
    cam = tiny.cameras[0]
    v = oracle.prepare_view(tiny.scene, cam, CFG)
    img, *_ = oracle.render(v, v["vals"], v["ranges"], cam, CFG)
    tg = (img + synth.target_noise(img.shape, 0.02, 1, 0)).astype(np.float32)
    d, _ = oracle.removal_effect(v, v["vals"], v["ranges"], cam, CFG, tg)
    m, im = oracle.removal_magnitude(v, v["vals"], v["ranges"], cam, CFG, tg)
    assert np.all(m >= np.abs(d) * (1 - 1e-12)) and np.count_nonzero(m) > 500
    per_splat = np.zeros_like(m)
    np.add.at(per_splat, v["vals"].astype(np.int64), im)
    assert np.allclose(per_splat, m, rtol=1e-12, atol=0)
    one = _scene(np.zeros((3, 1)), np.full((3, 1), -2.5), np.array([[1.0], [0], [0], [0]]), np.array([2.0]))
    c1 = synth.look_at_camera((0.0, 0.0, -3.0), 48, 40)
    v1 = oracle.prepare_view(one, c1, CFG)
    z = np.zeros((3, 40, 48), np.float32)
    d1, _ = oracle.removal_effect(v1, v1["vals"], v1["ranges"], c1, CFG, z)
    m1, _ = oracle.removal_magnitude(v1, v1["vals"], v1["ranges"], c1, CFG, z)
    assert d1[0] < 0 and m1[0] == pytest.approx(-4.0 * d1[0], rel=1e-12)
