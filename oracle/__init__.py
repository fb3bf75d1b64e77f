"""CPU oracle for the POTR removal-effect rasterizer -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library and its Python binding never import it, and the two
share no code: the oracle is ``potr_oracle.c`` (plain C, built with gcc, no contraction of
binary32 expressions) driven through ctypes from here.

Parity status per function (what pins it, see tests/test_oracle_*.py):

* ``exp2r``            -- against math.exp2 within the Taylor remainder bound; exactness on
                          integers; monotonicity on a dense grid.
* ``activate``         -- closed forms: axis-aligned quaternion gives diag(s^2); rotation
                          invariance of the trace; sigmoid at 0.
* ``project``          -- closed form of the 2D covariance for an axis-aligned splat on the
                          optical axis (f^2 sigma^2 / z^2 + lowpass); pinhole projection of the
                          centre; SH basis against scipy's complex spherical harmonics.
* ``bin`` / ranges     -- against numpy's stable argsort of the same keys; brute-force
                          enumeration of touched tiles.
* ``render``           -- one- and two-splat closed forms of Eq. (alpha blending); invariants
                          (T monotone, importance sums to 1 - T_final).
* ``removal_effect``   -- the definition (re-render without the splat, squared-error
                          difference) on the tiny scene with T_min = 0; one- and two-splat
                          closed forms of PD; zero effect of splats that never composite;
                          dSE = PD^2 >= 0 when the target is the render; the affine-in-alpha
                          identity PD_i = -alpha_i dc/dalpha_i checked by finite differences of
                          the definition.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "potr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile potr_oracle.c into oracle/_build/liboracle.so (gcc, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm", "-pthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Camera(C.Structure):
    _fields_ = [("w2c", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("near_z", C.c_float),
                ("lowpass", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_min", C.c_float)]


DEFAULTS = dict(tile_w=16, tile_h=16, near_z=0.2, lowpass=0.3, alpha_min=1.0 / 255.0,
                alpha_max=0.99, t_min=1e-4)


def make_config(**kw) -> Config:
    d = dict(DEFAULTS)
    d.update(kw)
    return Config(int(d["tile_w"]), int(d["tile_h"]), d["near_z"], d["lowpass"], d["alpha_min"],
                  d["alpha_max"], d["t_min"])


def make_camera(cam) -> Camera:
    c = Camera()
    for i in range(12):
        c.w2c[i] = float(cam.w2c[i])
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    return c


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, u32 = C.c_void_p, C.c_int64, C.c_uint32
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            L.orc_exp2r.restype = C.c_float
            L.orc_exp2r.argtypes = [C.c_float]
            L.orc_exp2r_array.argtypes = [i64, vp, vp]
            L.orc_exp2r_coeffs.argtypes = [vp]
            L.orc_activate.argtypes = [i64, vp, vp, vp, vp, vp]
            L.orc_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, vp]
            L.orc_project.argtypes = [i64, vp, vp, vp, vp, C.POINTER(Camera), C.POINTER(Config)] + [vp] * 9
            L.orc_bin.restype = i64
            L.orc_bin.argtypes = [i64, vp, vp, vp, vp, vp, vp, C.POINTER(Config), C.c_int32, C.c_uint64, u32, i64,
                                  vp, vp, vp, C.c_int32]
            L.orc_tile_hit.restype = C.c_int
            L.orc_tile_hit.argtypes = [C.c_float] * 6 + [C.c_int] * 4 + [C.c_float]
            L.orc_tile_ranges.argtypes = [i64, vp, C.c_uint64, i64, vp]
            L.orc_render.argtypes = [C.POINTER(Camera), C.POINTER(Config), i64, vp, vp, vp, vp, vp, vp,
                                     i64, vp, vp, vp, vp, vp]
            L.orc_removal_effect.argtypes = [C.POINTER(Camera), C.POINTER(Config), i64, vp, vp, vp, vp,
                                             vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_removal_magnitude.argtypes = [C.POINTER(Camera), C.POINTER(Config), i64, vp, vp, vp, vp,
                                                vp, vp, vp, vp, vp, vp]
            L.orc_pixel_lists.restype = i64
            L.orc_pixel_lists.argtypes = [C.POINTER(Camera), C.POINTER(Config), i64, vp, vp, vp, vp, vp, i64, vp,
                                          vp, vp]
            L.orc_removal_bruteforce.restype = C.c_double
            L.orc_removal_bruteforce.argtypes = [C.POINTER(Camera), C.POINTER(Config), i64, vp, vp, vp,
                                                 vp, vp, vp, vp, vp, i64]
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ------------------------------------------------------------------------------------------
# thin wrappers
# ------------------------------------------------------------------------------------------

def set_threads(n: int) -> None:
    """Threads over tiles for render and removal_effect (results do not depend on the count)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def exp2r(y) -> np.ndarray:
    y = _f32(np.atleast_1d(y))
    out = np.empty_like(y)
    lib().orc_exp2r_array(y.size, _p(y), _p(out))
    return out


def exp2r_coeffs() -> np.ndarray:
    out = np.empty(7, np.float32)
    lib().orc_exp2r_coeffs(_p(out))
    return out


def sh_basis(d) -> np.ndarray:
    out = np.empty(16, np.float64)
    lib().orc_sh_basis(float(d[0]), float(d[1]), float(d[2]), _p(out))
    return out


def activate(scene):
    n = scene.n
    ls, q, lg = _f32(scene.log_scales), _f32(scene.quats), _f32(scene.opacity_logits)
    cov = np.empty((6, n), np.float32)
    op = np.empty(n, np.float32)
    lib().orc_activate(n, _p(ls), _p(q), _p(lg), _p(cov), _p(op))
    return cov, op


def project(scene, cov3d, cam, cfg: Config, opacity) -> dict:
    """Projection of every splat into one view; the touched count is the number of tiles of the
    3-sigma rectangle that pass the tile test (alpha_min reachable at some pixel centre)."""
    n = scene.n
    opacity = _f32(opacity)
    means, sh = _f32(scene.means), _f32(scene.sh)
    out = dict(
        depth=np.empty(n, np.float32), mean2d=np.empty((2, n), np.float32),
        cov2d=np.empty((3, n), np.float32), conic=np.empty((3, n), np.float32),
        qcoef=np.empty((3, n), np.float32), radius=np.empty(n, np.float32),
        rect=np.empty((4, n), np.int32), touched=np.empty(n, np.uint32), rgb=np.empty((3, n), np.float64),
    )
    ccam = make_camera(cam)
    lib().orc_project(n, _p(means), _p(_f32(cov3d)), _p(opacity), _p(sh), C.byref(ccam), C.byref(cfg),
                      *[_p(out[k]) for k in ("depth", "mean2d", "cov2d", "conic", "qcoef", "radius",
                                             "rect", "touched", "rgb")])
    out["opacity"] = opacity
    return out


CULL_MAX_TILES = 64  # rectangles with more tiles keep every tile


def tile_hit(proj: dict, k: int, tx: int, ty: int, cfg: Config) -> bool:
    """The binning tile test for splat k and tile (tx, ty): True when some pixel centre of
    the tile can reach alpha >= alpha_min (conservative, binary32)."""
    m, q = proj["mean2d"], proj["qcoef"]
    return bool(lib().orc_tile_hit(float(m[0, k]), float(m[1, k]), float(q[0, k]), float(q[1, k]), float(q[2, k]),
                                   float(proj["opacity"][k]), int(tx), int(ty), cfg.tile_w, cfg.tile_h,
                                   float(cfg.alpha_min)))


def tiles_of(cam, cfg: Config):
    return (cam.width + cfg.tile_w - 1) // cfg.tile_w, (cam.height + cfg.tile_h - 1) // cfg.tile_h


def bin_sort(proj: dict, cam, cfg: Config, tile_base: int = 0, val_base: int = 0, whole_rect: bool = False):
    """Emit and stably sort the (tile, depth) keys; returns keys, vals, emit_index, ranges.

    ``whole_rect``: bin every tile of each splat's 3-sigma rectangle (the paper's footprint
    binning, no tile test) instead of only the tiles where alpha_min is reachable."""
    n = proj["depth"].size
    tx, ty = tiles_of(cam, cfg)
    if whole_rect:
        r = proj["rect"].astype(np.int64)
        m = int(((r[2] - r[0]) * (r[3] - r[1])).sum())
    else:
        m = int(proj["touched"].astype(np.int64).sum())
    keys = np.empty(max(m, 1), np.uint64)
    vals = np.empty(max(m, 1), np.uint32)
    emit = np.empty(max(m, 1), np.uint32)
    got = lib().orc_bin(n, _p(proj["touched"]), _p(proj["rect"]), _p(proj["depth"]), _p(proj["mean2d"]),
                        _p(proj["qcoef"]), _p(proj["opacity"]), C.byref(cfg), tx, tile_base, val_base, m,
                        _p(keys), _p(vals), _p(emit), int(bool(whole_rect)))
    assert got == m
    ranges = np.empty((tx * ty, 2), np.uint32)
    lib().orc_tile_ranges(m, _p(keys), tile_base, tx * ty, _p(ranges))
    return keys[:m], vals[:m], emit[:m], ranges


def render(proj: dict, vals, ranges, cam, cfg: Config, exclude: int = -1, tile_mask=None):
    n = proj["depth"].size
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W), np.float64)
    t32 = np.zeros((H, W), np.float32)
    t64 = np.zeros((H, W), np.float64)
    nl = np.zeros((H, W), np.uint32)
    ccam = make_camera(cam)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    lib().orc_render(C.byref(ccam), C.byref(cfg), n, _p(proj["mean2d"]), _p(proj["qcoef"]),
                     _p(proj["opacity"]), _p(proj["rgb"]), _p(vals), _p(ranges), exclude, _p(mask),
                     _p(img), _p(t32), _p(t64), _p(nl))
    return img, t32, t64, nl


def removal_effect(proj: dict, vals, ranges, cam, cfg: Config, target, tile_mask=None,
                   per_instance: bool = False):
    """Per-splat dSSE (sum over pixels and channels of dSE) and importance sums for one view."""
    n = proj["depth"].size
    ccam = make_camera(cam)
    dsse = np.zeros(n, np.float64)
    imp = np.zeros(n, np.float64)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    tgt = _f32(target)
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    idse = np.zeros(max(vals.size, 1), np.float64) if per_instance else None
    iimp = np.zeros(max(vals.size, 1), np.float64) if per_instance else None
    lib().orc_removal_effect(C.byref(ccam), C.byref(cfg), n, _p(proj["mean2d"]), _p(proj["qcoef"]),
                             _p(proj["opacity"]), _p(proj["rgb"]), _p(vals), _p(ranges), _p(tgt),
                             _p(mask), _p(dsse), _p(imp), _p(idse), _p(iimp))
    if per_instance:
        return dsse, imp, idse[: vals.size], iimp[: vals.size]
    return dsse, imp


def removal_magnitude(proj: dict, vals, ranges, cam, cfg: Config, target, tile_mask=None):
    """(per splat, per instance) sums of the magnitudes of the terms each dSE is formed from:
    the rounding scale of a binary32 evaluation (a tolerance quantity, not the method)."""
    n = proj["depth"].size
    ccam = make_camera(cam)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8)
    mag = np.zeros(n, np.float64)
    imag = np.zeros(max(vals.size, 1), np.float64)
    lib().orc_removal_magnitude(C.byref(ccam), C.byref(cfg), n, _p(proj["mean2d"]), _p(proj["qcoef"]),
                                _p(proj["opacity"]), _p(proj["rgb"]), _p(vals), _p(ranges), _p(_f32(target)),
                                _p(mask), _p(mag), _p(imag))
    return mag, imag[: vals.size]


def removal_bruteforce(proj: dict, vals, ranges, cam, cfg: Config, target, image, k: int) -> float:
    n = proj["depth"].size
    ccam = make_camera(cam)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    return lib().orc_removal_bruteforce(C.byref(ccam), C.byref(cfg), n, _p(proj["mean2d"]),
                                        _p(proj["qcoef"]), _p(proj["opacity"]), _p(proj["rgb"]),
                                        _p(vals), _p(ranges), _p(_f32(target)),
                                        _p(np.ascontiguousarray(image, np.float64)), k)


def pixel_lists(proj: dict, vals, ranges, cam, cfg: Config):
    """Composited (pixel, splat, list position) triples of one view, in compositing order."""
    n = proj["depth"].size
    ccam = make_camera(cam)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    cap = max(1, min(int(vals.size) * cfg.tile_w * cfg.tile_h, 1 << 26))
    while True:
        pix = np.empty(cap, np.int64)
        k = np.empty(cap, np.uint32)
        pos = np.empty(cap, np.uint32)
        m = lib().orc_pixel_lists(C.byref(ccam), C.byref(cfg), n, _p(proj["mean2d"]), _p(proj["qcoef"]),
                                  _p(proj["opacity"]), _p(vals), _p(ranges), cap, _p(pix), _p(k), _p(pos))
        if m >= 0:
            return pix[:m], k[:m], pos[:m]
        cap = -m


# ------------------------------------------------------------------------------------------
# whole-view helpers
# ------------------------------------------------------------------------------------------

def prepare_view(scene, cam, cfg: Config, act=None) -> dict:
    """Activation + projection + binning of one view; returns a dict of every stage's output."""
    cov, op = act if act is not None else activate(scene)
    proj = project(scene, cov, cam, cfg, op)
    proj["cov3d"] = cov
    keys, vals, emit, ranges = bin_sort(proj, cam, cfg)
    proj.update(keys=keys, vals=vals, emit=emit, ranges=ranges)
    return proj


def view_dsse(scene, cam, cfg: Config, target, act=None):
    """dSSE_k(s) = sum_x sum_ch dSE_k and sum_x T alpha for every splat, one view."""
    v = prepare_view(scene, cam, cfg, act)
    return removal_effect(v, v["vals"], v["ranges"], cam, cfg, target)


def dmse(scene, cams, cfg: Config, targets):
    """dMSE_k = (1/N) sum_s (1/P_s) sum_x (1/3) dSE_k and I_k = (1/N) sum_s (1/P_s) sum_x T alpha.

    Views are added in order, each view's contribution divided by 3 P_s and by N first.
    """
    act = activate(scene)
    n_views = len(cams)
    out = np.zeros(scene.n, np.float64)
    imp = np.zeros(scene.n, np.float64)
    for cam, tgt in zip(cams, targets):
        d, i = view_dsse(scene, cam, cfg, tgt, act)
        out += d / (3.0 * cam.pixels) / n_views
        imp += i / float(cam.pixels) / n_views
    return out, imp
