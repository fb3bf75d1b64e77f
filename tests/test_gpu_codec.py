"""The encoder on the device (potr_codec_encode) against the codec oracle: the raw bitstreams
must be equal byte for byte (octree node bytes, leaf order, quantised attributes)."""
import numpy as np
import pytest

import synth
from oracle import codec as ocodec

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
