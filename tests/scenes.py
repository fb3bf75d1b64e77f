"""Hand-built test scenes shared by the oracle pins and the device parity tests."""
import numpy as np

import synth


def clamp_scene(cam, seed: int = 41):
    """300 random splats plus three large isotropic splats at camera-space x / z = 1.5, -1.6 and
    1.75, z = 3 (beyond the Jacobian clamp, 1.3 times the half field of view: 0.75 for a 64-pixel
    wide view with a 60 degree field) whose footprints reach into the image; splats 0-39 nearly
    opaque (opacity 0.9997: alpha clamped to alpha_max at their centres) and splats 40-79 with a
    red SH DC of -3 (colour clamped at 0).  Returns (scene, number of splats beyond the clamp)."""
    base = synth.uniform_cube_scene(300, seed)
    W = cam.w2c.reshape(3, 4).astype(np.float64)
    pts = np.array([[s * r * 3.0, 0.2 * j, 3.0] for j, (s, r) in enumerate([(1, 1.5), (-1, 1.6), (1, 1.75)])])
    far = W[:, :3].T @ (pts.T - W[:, 3:4])  # x_c = R x + t  ->  x = R^T (x_c - t)
    m = far.shape[1]
    sh_far = np.zeros((16, 3, m), np.float32)
    sh_far[0] = 0.8
    sc = synth.Scene(
        np.concatenate([base.means, far.astype(np.float32)], axis=1),
        np.concatenate([base.log_scales, np.full((3, m), 0.2, np.float32)], axis=1),
        np.concatenate([base.quats, np.tile(np.array([[1.0], [0.0], [0.0], [0.0]], np.float32), m)], axis=1),
        np.concatenate([base.opacity_logits, np.full(m, 2.0, np.float32)]),
        np.concatenate([base.sh, sh_far], axis=2),
    )
    sc.opacity_logits[:40] = 8.0
    sc.sh[0, 0, 40:80] = -3.0
    return sc, m
