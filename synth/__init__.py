"""Seeded synthetic scenes, cameras and target-noise for the removal-effect workloads.

This module holds input generation only: splat parameter draws, camera poses and the
random perturbations used to build target images. It contains none of the method's
arithmetic (no activation, projection, compositing or removal effect), so both the CPU
oracle and the CUDA path may take their inputs from here.

Workloads (all fp32, parameters stored as SoA planes):

* ``tiny``      1,000 splats, one 128x128 view at radius 3 (the paper's method on a toy scene).
* ``scene``     1M splats (70 % in the unit ball, 30 % in a 2..10 shell), 16 views 1280x720.
* ``batched``   3M splats, 200 views of mixed resolution {960x540, 1280x720, 1920x1080}.
* ``grad``      1M splats, 8 views 1280x720 (forward + backward workload).
* ``large``     6M splats, 300 views 1920x1080, shell outer radius 20.

Splat parameter distributions follow the scene sizes the paper evaluates (0.3M-6M splats,
Section V): log-scales N(-4, 0.5) per axis, quaternions normalised N(0,1)^4 with the real
part first, opacity logits N(0, 1.5), SH degree 3 with DC ~ N(0, 0.5) and the 45 AC
coefficients ~ N(0, 0.05).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SH_COEFFS = 16  # degree 3: (3 + 1)^2 basis functions per colour channel


@dataclass
class Scene:
    """Splat parameters as SoA planes (float32).

    means[3][N], log_scales[3][N], quats[4][N] (w, x, y, z), opacity_logits[N],
    sh[16][3][N] (coefficient-major, DC first, channels R, G, B).
    """

    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.means.shape[1])

    def subset(self, keep: np.ndarray) -> "Scene":
        """Scene restricted to the splats where ``keep`` is true (order kept)."""
        return Scene(
            np.ascontiguousarray(self.means[:, keep]),
            np.ascontiguousarray(self.log_scales[:, keep]),
            np.ascontiguousarray(self.quats[:, keep]),
            np.ascontiguousarray(self.opacity_logits[keep]),
            np.ascontiguousarray(self.sh[:, :, keep]),
        )


@dataclass
class Camera:
    """Pinhole camera: world-to-camera rows [R | t] (3x4, row-major), intrinsics, size.

    Camera space looks along +z with +y pointing down the image; pixel (x, y) has its
    centre at (x + 0.5, y + 0.5).
    """

    w2c: np.ndarray  # float32 (12,)
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def pixels(self) -> int:
        return self.width * self.height


@dataclass
class Workload:
    name: str
    scene: Scene
    cameras: list
    seed: int
    # Per-view target recipe: drop fraction of splats and Gaussian noise sigma.
    target_drop: float = 0.0
    target_noise: float = 0.0
    extra: dict = field(default_factory=dict)


def _draw_params(rng: np.random.Generator, means: np.ndarray) -> Scene:
    n = means.shape[1]
    log_scales = rng.normal(-4.0, 0.5, size=(3, n)).astype(np.float32)
    q = rng.normal(0.0, 1.0, size=(4, n))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    opacity_logits = rng.normal(0.0, 1.5, size=n).astype(np.float32)
    sh = np.empty((SH_COEFFS, 3, n), dtype=np.float32)
    sh[0] = rng.normal(0.0, 0.5, size=(3, n))
    sh[1:] = rng.normal(0.0, 0.05, size=(SH_COEFFS - 1, 3, n))
    return Scene(
        np.ascontiguousarray(means.astype(np.float32)),
        log_scales,
        np.ascontiguousarray(q.astype(np.float32)),
        opacity_logits,
        sh,
    )


def _uniform_ball(rng: np.random.Generator, n: int, r_in: float, r_out: float) -> np.ndarray:
    """Points uniform in volume in the spherical shell r_in <= r <= r_out."""
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0, keepdims=True)
    u = rng.uniform(size=n)
    r = np.cbrt(r_in ** 3 + u * (r_out ** 3 - r_in ** 3))
    return d * r


def uniform_cube_scene(n: int, seed: int) -> Scene:
    """Means uniform in [-1, 1]^3 with the standard parameter distributions."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(3, n))
    return _draw_params(rng, means)


def ball_shell_scene(n: int, seed: int, shell_outer: float = 10.0) -> Scene:
    """70 % of the means uniform in the unit ball, 30 % uniform in the shell 2..shell_outer."""
    rng = np.random.default_rng(seed)
    n_ball = int(round(0.7 * n))
    means = np.concatenate(
        [_uniform_ball(rng, n_ball, 0.0, 1.0), _uniform_ball(rng, n - n_ball, 2.0, shell_outer)], axis=1
    )
    perm = rng.permutation(n)
    return _draw_params(rng, means[:, perm])


def look_at_camera(position, width: int, height: int, vfov_deg: float = 60.0) -> Camera:
    """Camera at ``position`` looking at the origin, world up +y, vertical field of view."""
    p = np.asarray(position, dtype=np.float64)
    fwd = -p / np.linalg.norm(p)
    down = np.array([0.0, -1.0, 0.0])
    x = np.cross(down, fwd)
    x /= np.linalg.norm(x)
    y = np.cross(fwd, x)
    rot = np.stack([x, y, fwd])  # rows: camera axes in world coordinates
    t = -rot @ p
    w2c = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32).reshape(-1)
    fy = (0.5 * height) / math.tan(math.radians(0.5 * vfov_deg))
    return Camera(w2c, float(fy), float(fy), 0.5 * width, 0.5 * height, int(width), int(height))


def ring_cameras(
    n_views: int,
    radius,
    heights,
    sizes,
    vfov_deg: float = 60.0,
) -> list:
    """Cameras evenly spaced in angle on a ring in the x-z plane, looking at the origin."""
    cams = []
    for i in range(n_views):
        th = 2.0 * math.pi * i / n_views
        r = float(radius[i]) if np.ndim(radius) else float(radius)
        h = float(heights[i]) if np.ndim(heights) else float(heights)
        w, hh = sizes[i] if isinstance(sizes, list) else sizes
        cams.append(look_at_camera((r * math.cos(th), h, r * math.sin(th)), w, hh, vfov_deg))
    return cams


SIZES_MIXED = [(960, 540), (1280, 720), (1920, 1080)]


def workload(name: str, n_override: int | None = None, views_override: int | None = None) -> Workload:
    """Build one of the named workloads (seeded: tiny 1000, scene 1001, batched 1002, grad 1003, large 1004)."""
    if name == "tiny":
        seed = 1000
        n = n_override or 1000
        scene = uniform_cube_scene(n, seed)
        cams = [look_at_camera((0.0, 0.0, -3.0), 128, 128)]
        return Workload(name, scene, cams, seed, 0.0, 0.02)
    if name in ("scene", "grad"):
        seed = 1001 if name == "scene" else 1003
        n = n_override or 1_000_000
        v = views_override or (16 if name == "scene" else 8)
        scene = ball_shell_scene(n, seed)
        rng = np.random.default_rng(seed + 7)
        heights = rng.uniform(-0.5, 0.5, size=v)
        cams = ring_cameras(v, 4.0, heights, (1280, 720))
        if name == "scene":
            return Workload(name, scene, cams, seed, 0.05, 0.01)
        return Workload(name, scene, cams, seed, 0.0, 0.01)
    if name == "batched":
        seed = 1002
        n = n_override or 3_000_000
        v = views_override or 200
        scene = ball_shell_scene(n, seed)
        rng = np.random.default_rng(seed + 7)
        radii = rng.uniform(3.0, 6.0, size=v)
        heights = rng.uniform(-0.5, 0.5, size=v)
        sizes = [SIZES_MIXED[i] for i in rng.integers(0, 3, size=v)]
        cams = ring_cameras(v, radii, heights, sizes)
        return Workload(name, scene, cams, seed, 0.05, 0.01)
    if name == "large":
        seed = 1004
        n = n_override or 6_000_000
        v = views_override or 300
        scene = ball_shell_scene(n, seed, shell_outer=20.0)
        rng = np.random.default_rng(seed + 7)
        heights = rng.uniform(-0.5, 0.5, size=v)
        cams = ring_cameras(v, 4.0, heights, (1920, 1080))
        return Workload(name, scene, cams, seed, 0.05, 0.01)
    raise ValueError(f"unknown workload {name!r}")


def target_drop_mask(n: int, frac: float, seed: int) -> np.ndarray:
    """Boolean keep-mask that drops a seeded random ``frac`` of the splats."""
    rng = np.random.default_rng(seed + 11)
    return rng.uniform(size=n) >= frac


def target_noise(shape, sigma: float, seed: int, view: int) -> np.ndarray:
    """Seeded Gaussian noise image (float32) added to a rendered target."""
    rng = np.random.default_rng([seed, 13, view])
    return rng.normal(0.0, sigma, size=shape).astype(np.float32)


def cameras_to_array(cams) -> np.ndarray:
    """Pack cameras as the C record {float w2c[12], fx, fy, cx, cy; int32 width, height} (18 x 4 bytes)."""
    rec = np.zeros((len(cams), 18), dtype=np.float32)
    for i, c in enumerate(cams):
        rec[i, :12] = c.w2c
        rec[i, 12:16] = (c.fx, c.fy, c.cx, c.cy)
        rec[i, 16:18] = np.array([c.width, c.height], dtype=np.int32).view(np.float32)
    return rec
