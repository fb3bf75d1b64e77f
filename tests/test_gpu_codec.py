"""The codec on the device against the codec oracle: the encoder's raw bitstream must equal the
oracle's byte for byte (node bytes, shared-leaf table, leaf order, quantised attributes); the
decoder's scene must equal the oracle's decode (positions, scales, rotations, SH exactly as
float32 of the binary64 values; opacity logits to float32 rounding); malformed streams are
reported through the status word; and a POTR-FT cycle recovers quality lost to pruning."""
import numpy as np
import pytest

import synth
from oracle import codec as ocodec
from oracle.sh_compact import camera_centre

pytestmark = pytest.mark.gpu

EYES = np.array([[3.0, 0.2, 0.0], [-2.0, 0.0, 2.5], [0.0, 3.0, -0.5]])


def _scene(n, seed):
    sc = synth.uniform_cube_scene(n, seed)
    if n >= 20:
        sc.means[:, 7] = sc.means[:, 3]   # coincident splats: a shared leaf at the depth limit
        sc.means[:, 11] = sc.means[:, 3]
        sc.quats[:, 5] = -sc.quats[:, 5]  # w < 0: the stored quaternion flips sign
    return sc


def _first_difference(a: bytes, b: bytes):
    for i, (x, y) in enumerate(zip(a, b)):
        if x != y:
            return i
    return min(len(a), len(b)) if len(a) != len(b) else None


@pytest.mark.parametrize("n,q", [(2, 0.5), (17, 0.5), (3000, 0.5), (3000, 0.9), (60000, 0.3)])
def test_device_bitstream_equals_oracle(n, q):
    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.codec import encode, params
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    sc = _scene(n, 40 + n)
    p = params(q)
    want = ocodec.encode(sc, EYES, p=ocodec.params(q))
    got = encode(scene_to_device(sc), EYES, p=p)
    assert np.array_equal(got["order"], want["order"])
    i = _first_difference(got["raw"], want["raw"])
    assert i is None, f"streams differ from byte {i} (node bytes end at {80 + len(want['occupancy'])})"
    if n >= 20:
        d = ocodec.decode(got["compressed"])
        o = want["order"]
        mu = sc.means[:, o].astype(np.float64)
        pp = ocodec.params(q)
        tol = ocodec.tolerance(mu, EYES, pp["beta"], pp["gamma"])
        err = np.linalg.norm(d["means"] - mu, axis=0)
        shared = d["depths"] == ocodec.DEPTH
        assert np.all(err[~shared] < tol[~shared]) and shared.sum() >= 3


def _decode_matches(dev_scene, want, n):
    got = {k: t.cpu().numpy() for k, t in dev_scene.items()}
    for k in ("means", "log_scales", "quats"):
        assert np.array_equal(got[k], want[k].astype(np.float32)), k
    assert np.array_equal(got["sh"], want["sh"].astype(np.float32))
    np.testing.assert_allclose(got["opacity_logits"], want["opacity_logits"], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("n,q", [(1, 0.5), (2, 0.5), (17, 0.5), (3000, 0.5), (3000, 0.9), (60000, 0.3)])
def test_device_decode_equals_oracle(n, q):
    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.codec import decode

    build.build()
    sc = _scene(n, 70 + n)
    want_enc = ocodec.encode(sc, EYES, p=ocodec.params(q))
    want = ocodec.decode(want_enc["compressed"])
    if n >= 20:
        assert want["n_dups"] >= 1
    got = decode(want_enc["compressed"])
    _decode_matches(got, want, n)


def test_device_roundtrip_equals_the_decode_of_the_stream():
    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.codec import roundtrip
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    sc = _scene(20000, 5)
    want_enc = ocodec.encode(sc, EYES, p=ocodec.params(0.5))
    want = ocodec.decode(want_enc["compressed"])
    got, order = roundtrip(scene_to_device(sc), EYES, q=0.5)
    assert np.array_equal(order.cpu().numpy(), want_enc["order"])
    _decode_matches(got, want, sc.n)


def _corrupt_status(nodes: bytes, dups, n, attrs_n=None):
    import torch

    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300.codec import Decoder

    dev = torch.device("cuda")
    t_nodes = torch.as_tensor(np.frombuffer(nodes, np.uint8).copy(), device=dev)
    t_dups = torch.as_tensor(np.array(dups, np.int32).reshape(-1), device=dev) if len(dups) else None
    attrs = torch.zeros(55 * (attrs_n or n), dtype=torch.int32, device=dev)
    dec = Decoder(len(nodes), n, dev)
    p = {"sf_scale": 2001.0, "sf_rotation": 201.0, "sf_opacity": 101.0, "sf_sh": 51.0}
    dec.run(t_nodes, t_dups, len(dups), attrs, (0.0, 0.0, 0.0, 1.0), p)
    torch.cuda.synchronize()
    return int(dec.status[0].item()), B


def test_malformed_streams_are_reported():
    # the three-splat stream of the oracle pins: root 0x81, 20 single-child bytes and a shared
    # leaf (ordinal 0, one extra splat), then three single-child bytes and a leaf
    good = bytes([0x81] + [0x01] * 20 + [0x00] + [0x80] * 3 + [0x00])
    code, B = _corrupt_status(good, [(0, 1)], 3)
    assert code == B.POTR_OK
    # a leaf that claims a child: the tree never closes
    code, _ = _corrupt_status(good[:-1] + bytes([0x01]), [(0, 1)], 3)
    assert code == B.POTR_ERR_CORRUPT
    # a byte too many: the tree closes before the stream ends
    code, _ = _corrupt_status(good + bytes([0x00]), [(0, 1)], 3)
    assert code == B.POTR_ERR_CORRUPT
    # the table names a leaf that does not exist
    code, _ = _corrupt_status(good, [(5, 1)], 3)
    assert code == B.POTR_ERR_CORRUPT
    # leaves and table do not account for n splats
    code, _ = _corrupt_status(good, [(0, 1)], 4)
    assert code == B.POTR_ERR_CORRUPT
    # a path below the depth limit (22 single-child levels)
    deep = bytes([0x01] * 22 + [0x00])
    code, _ = _corrupt_status(deep, [], 1)
    assert code == B.POTR_ERR_CORRUPT


def _loss(scene, rec, targets, cfg):
    import torch

    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame

    tot = 0.0
    for v, tgt in enumerate(targets):
        f = RemovalEffectFrame(scene, rec[v:v + 1], with_importance=False, **cfg)
        f.plan(1.5)
        img = f.image_buffer()
        f.render(img)
        tot += float(torch.mean((img - tgt) ** 2).item())
    return tot / len(targets)


def test_potr_ft_cycle_recovers_quality_lost_to_pruning():
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.codec import decode, roundtrip
    from paper_2601_14821_gb300.finetune import potr_ft
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    build.build()
    sc = synth.uniform_cube_scene(4000, 29)
    cams = synth.ring_cameras(6, 3.0, 0.3, (128, 96))
    rec = synth.cameras_to_array(cams)
    eyes = np.array([camera_centre(c) for c in cams])
    cfg = dict(tile_w=16, tile_h=16, batch=256)
    full = scene_to_device(sc)
    targets = []
    for v in range(len(cams)):
        f = RemovalEffectFrame(full, rec[v:v + 1], with_importance=False, **cfg)
        f.plan()
        img = f.image_buffer()
        f.render(img)
        targets.append(img.clone())
    torch.cuda.synchronize()
    keep = torch.from_numpy(np.random.default_rng(0).random(sc.n) < 0.7).cuda()
    pruned = {k: t[..., keep].contiguous() for k, t in full.items()}
    before, _ = roundtrip(pruned, eyes, q=0.5)
    l0 = _loss(before, rec, targets, cfg)
    out = potr_ft(pruned, rec, targets, eyes, q=0.5, cycles=2, iterations=150, extent=3.0, **cfg)
    after = decode(out["compressed"])
    l1 = _loss(after, rec, targets, cfg)
    assert len(out["losses"]) == 2 and l1 < 0.8 * l0, (l0, l1)
