"""ctypes binding of libpotr (include/potr.h): same names, argument marshalling only.

Every compute step runs in the CUDA library; this module converts torch tensors to device
pointers, Python values to the C structs, and C status codes to exceptions.  It raises
when the library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpotr.so")
_lock = threading.Lock()
_lib = None

POTR_OK = 0
POTR_ERR_INVALID_ARGUMENT = 1
POTR_ERR_CUDA = 2
POTR_ERR_CAPACITY = 3
POTR_ERR_TIMEOUT = 4
POTR_ERR_NUMERIC = 5
POTR_ERR_UNSUPPORTED = 6
POTR_ERR_TOO_LARGE = 7
POTR_ERR_CORRUPT = 8
POTR_STATIC_MAX_INSTANCES = 4194304
POTR_STATIC_MAX_VIEW_SPLATS = 1048576


class PotrError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status_string(status)} ({status})")
        self.status = status


class Scene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64)]


class Camera(C.Structure):
    _fields_ = [("w2c", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class RasterConfig(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("batch", C.c_int32), ("near_z", C.c_float),
                ("lowpass", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float)]


class ViewInfo(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32),
                ("tile_base", C.c_int64), ("pixel_base", C.c_int64)]


class Frame(C.Structure):
    _fields_ = [("cams", C.c_void_p), ("info", C.c_void_p), ("n_views", C.c_int32), ("total_tiles", C.c_int64),
                ("total_pixels", C.c_int64)]


class Views(C.Structure):
    _fields_ = [("cov3d", C.c_void_p), ("opacity", C.c_void_p), ("raster", C.c_void_p), ("depth", C.c_void_p),
                ("rect", C.c_void_p), ("touched", C.c_void_p), ("offsets", C.c_void_p),
                ("n_instances", C.c_void_p), ("cull", C.c_void_p)]


class SceneGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class CodecParams(C.Structure):
    _fields_ = [("sf_scale", C.c_double), ("sf_rotation", C.c_double), ("sf_opacity", C.c_double),
                ("sf_sh", C.c_double), ("beta", C.c_double), ("gamma", C.c_double)]


class DeviceStatus(C.Structure):
    _fields_ = [("code", C.c_int32), ("n_nonfinite", C.c_int32), ("required_instances", C.c_int64)]


# Every exported symbol of include/potr.h, with its ctypes signature.
_P, _I32, _I64, _SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
SIGNATURES = {
    "potr_status_string": (C.c_char_p, [_I32]),
    "potr_version": (_I32, []),
    "potr_view_layout": (_I32, [_P, _I32, C.POINTER(RasterConfig), _P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "potr_preprocess": (_I32, [C.POINTER(Scene), C.POINTER(Frame), C.POINTER(RasterConfig), C.POINTER(Views), _P,
                               _P]),
    "potr_bin_sort_workspace_size": (_SZ, [_I64, _I32, _I64, _I64]),
    "potr_bin_sort": (_I32, [C.POINTER(Views), C.POINTER(Frame), C.POINTER(RasterConfig), _I64, _I64, _P, _P, _P,
                             _P, _P, _SZ, _P]),
    "potr_render": (_I32, [C.POINTER(Views), C.POINTER(Frame), C.POINTER(RasterConfig), _I64, _P, _P, _P, _P, _P,
                           _P, _P]),
    "potr_removal_workspace_size": (_SZ, [_I64, _I64, _I32]),
    "potr_removal_effect": (_I32, [C.POINTER(Views), C.POINTER(Frame), C.POINTER(RasterConfig), _I64, _P, _P, _P,
                                   _P, _I32, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "potr_tile_schedule_workspace_size": (_SZ, []),
    "potr_tile_schedule": (_I32, [C.POINTER(Frame), _P, _P, _P, _SZ, _P]),
    "potr_pair_stats": (_I32, [C.POINTER(Views), C.POINTER(Frame), C.POINTER(RasterConfig), _I64, _P, _P, _P, _P]),
    "potr_launch_count": (C.c_uint64, []),
    "potr_time_next_tile_kernel": (_I32, [_P, _P]),
    "potr_selftest_wait_timeout": (_I32, [_P, _SZ, _I32, _P, _P]),
    "potr_loss_workspace_size": (_SZ, [_I64]),
    "potr_loss_grad": (_I32, [C.POINTER(Frame), _P, _P, C.c_float, _P, _P, _P, _SZ, _P]),
    "potr_render_backward_workspace_size": (_SZ, [_I64, _I64]),
    "potr_render_backward": (_I32, [C.POINTER(Scene), C.POINTER(Views), C.POINTER(Frame), C.POINTER(RasterConfig), _P,
                                    _P, _P, _P, _P, _P, _I64, C.POINTER(SceneGrads), _P, _SZ, _P]),
    "potr_bin_sort_static": (_I32, [C.POINTER(Views), C.POINTER(Frame), C.POINTER(RasterConfig), _I64, _I64, _P, _P,
                                    _P, _P, _P]),
    "potr_prune_workspace_size": (_SZ, [_I64]),
    "potr_prune_select": (_I32, [_I64, _P, _P, _P, C.c_double, C.c_double, _I32, _P, _P, _SZ, _P]),
    "potr_prune_apply": (_I32, [_I64, _P, _P, _P]),
    "potr_sh_compact": (_I32, [C.POINTER(Scene), C.POINTER(Frame), _P, C.c_double, C.c_double, C.c_double, _P, _P,
                               _P, _P]),
    "potr_codec_workspace_size": (_SZ, [_I64]),
    "potr_codec_encode": (_I32, [C.POINTER(Scene), _P, _I32, C.POINTER(CodecParams), _P, _P, _P, _P, _P, _P, _P, _P,
                                 _P, _SZ, _P]),
    "potr_codec_decode_workspace_size": (_SZ, [_I64, _I64]),
    "potr_codec_decode": (_I32, [_P, _I64, _P, _I64, _P, _I64, C.POINTER(C.c_double), C.POINTER(CodecParams),
                                 C.POINTER(SceneGrads), _P, _P, _SZ, _P]),
    "potr_adam_step": (_I32, [C.POINTER(SceneGrads), C.POINTER(SceneGrads), C.POINTER(SceneGrads),
                              C.POINTER(SceneGrads), _I64, _I64, C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float,
                              _P]),
    "potr_adam_schedule": (_I32, [_I64, _I64, C.POINTER(C.c_float), C.c_float, C.c_float, _P]),
    "potr_adam_step_scheduled": (_I32, [C.POINTER(SceneGrads), C.POINTER(SceneGrads), C.POINTER(SceneGrads),
                                        C.POINTER(SceneGrads), _I64, _P, _I64, _P, C.c_float, C.c_float, C.c_float,
                                        _P]),
}


def lib():
    """Load libpotr.so (built by ``paper_2601_14821_gb300.build``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpotr.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().potr_status_string(int(status)).decode()


def _check(fn: str, status: int):
    if status != POTR_OK:
        raise PotrError(fn, status)


def ptr(t) -> int | None:
    """Device (or host) address of a torch tensor / numpy array, None for None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def stream_handle(stream=None) -> int | None:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


DEFAULT_CONFIG = dict(tile_w=16, tile_h=16, batch=256, near_z=0.2, lowpass=0.3, alpha_min=1.0 / 255.0,
                      alpha_max=0.99, t_min=1e-4)


def make_config(**kw) -> RasterConfig:
    d = dict(DEFAULT_CONFIG)
    d.update(kw)
    return RasterConfig(int(d["tile_w"]), int(d["tile_h"]), int(d["batch"]), d["near_z"], d["lowpass"],
                        d["alpha_min"], d["alpha_max"], d["t_min"])


# ------------------------------------------------------------------------------------------
# the C entry points
# ------------------------------------------------------------------------------------------

def potr_view_layout(cams_rec: np.ndarray, cfg: RasterConfig):
    """cams_rec: (V, 18) float32 camera records.  Returns (info (V,) ViewInfo array as
    uint8 bytes, total_tiles, total_pixels)."""
    cams_rec = np.ascontiguousarray(cams_rec, np.float32)
    v = cams_rec.shape[0]
    info = np.zeros(v * C.sizeof(ViewInfo), np.uint8)
    tt, tp = C.c_int64(0), C.c_int64(0)
    _check("potr_view_layout", lib().potr_view_layout(cams_rec.ctypes.data, v, C.byref(cfg), info.ctypes.data,
                                                      C.byref(tt), C.byref(tp)))
    return info, tt.value, tp.value


def potr_preprocess(scene: Scene, frame: Frame, cfg: RasterConfig, views: Views, stream=None, status=None):
    _check("potr_preprocess", lib().potr_preprocess(C.byref(scene), C.byref(frame), C.byref(cfg), C.byref(views),
                                                    ptr(status), stream_handle(stream)))


def potr_bin_sort_workspace_size(n: int, n_views: int, total_tiles: int, capacity: int) -> int:
    return int(lib().potr_bin_sort_workspace_size(n, n_views, total_tiles, capacity))


def potr_bin_sort(views: Views, frame: Frame, cfg: RasterConfig, n: int, capacity: int, tiles, vals, ranges, status,
                  ws, stream=None):
    _check("potr_bin_sort", lib().potr_bin_sort(C.byref(views), C.byref(frame), C.byref(cfg), n, capacity, ptr(tiles),
                                                ptr(vals), ptr(ranges), ptr(status), ptr(ws), ws.numel(),
                                                stream_handle(stream)))


def potr_render(views: Views, frame: Frame, cfg: RasterConfig, n: int, vals, ranges, images=None, t_final=None,
                n_last=None, stream=None, order=None):
    _check("potr_render", lib().potr_render(C.byref(views), C.byref(frame), C.byref(cfg), n, ptr(vals), ptr(ranges),
                                            ptr(order), ptr(images), ptr(t_final), ptr(n_last),
                                            stream_handle(stream)))


def potr_removal_workspace_size(capacity: int, total_tiles: int, with_importance: bool) -> int:
    return int(lib().potr_removal_workspace_size(capacity, total_tiles, 1 if with_importance else 0))


def potr_removal_effect(views: Views, frame: Frame, cfg: RasterConfig, n: int, vals, ranges, targets,
                        n_views_total: int, capacity: int, inst_dse, inst_imp=None, dmse=None, importance=None,
                        dsse_view=None, images=None, stream=None, order=None, imp_view=None, ws=None):
    _check("potr_removal_effect",
           lib().potr_removal_effect(C.byref(views), C.byref(frame), C.byref(cfg), n, ptr(vals), ptr(ranges),
                                     ptr(order), ptr(targets), n_views_total, capacity, ptr(inst_dse), ptr(inst_imp),
                                     ptr(dmse), ptr(importance), ptr(dsse_view), ptr(imp_view), ptr(images),
                                     ptr(ws), 0 if ws is None else ws.numel(), stream_handle(stream)))


def potr_tile_schedule_workspace_size() -> int:
    return int(lib().potr_tile_schedule_workspace_size())


def potr_tile_schedule(frame: Frame, ranges, order, ws, stream=None):
    _check("potr_tile_schedule", lib().potr_tile_schedule(C.byref(frame), ptr(ranges), ptr(order), ptr(ws), ws.numel(),
                                                          stream_handle(stream)))


def potr_pair_stats(views: Views, frame: Frame, cfg: RasterConfig, n: int, vals, ranges, counts, stream=None):
    _check("potr_pair_stats", lib().potr_pair_stats(C.byref(views), C.byref(frame), C.byref(cfg), n, ptr(vals),
                                                    ptr(ranges), ptr(counts), stream_handle(stream)))


def potr_launch_count() -> int:
    return int(lib().potr_launch_count())


def potr_bin_sort_static(views: Views, frame: Frame, cfg: RasterConfig, n: int, capacity: int, tiles, vals, ranges,
                         status, stream=None):
    """potr_bin_sort with the library's fixed scratch instead of a caller workspace."""
    _check("potr_bin_sort_static", lib().potr_bin_sort_static(C.byref(views), C.byref(frame), C.byref(cfg), n,
                                                              capacity, ptr(tiles), ptr(vals), ptr(ranges),
                                                              ptr(status), stream_handle(stream)))


def potr_loss_workspace_size(total_pixels: int) -> int:
    return int(lib().potr_loss_workspace_size(total_pixels))


def potr_loss_grad(frame: Frame, images, targets, lam: float, loss, dL_dimages, ws, stream=None):
    _check("potr_loss_grad", lib().potr_loss_grad(C.byref(frame), ptr(images), ptr(targets), lam, ptr(loss),
                                                  ptr(dL_dimages), ptr(ws), 0 if ws is None else ws.numel(),
                                                  stream_handle(stream)))


def potr_render_backward_workspace_size(capacity: int, n_view_splats: int) -> int:
    return int(lib().potr_render_backward_workspace_size(capacity, n_view_splats))


def potr_render_backward(scene: Scene, views: Views, frame: Frame, cfg: RasterConfig, vals, ranges, t_final, n_last,
                         dL_dimages, capacity: int, grads: SceneGrads, ws, stream=None, order=None):
    _check("potr_render_backward",
           lib().potr_render_backward(C.byref(scene), C.byref(views), C.byref(frame), C.byref(cfg), ptr(vals),
                                      ptr(ranges), ptr(order), ptr(t_final), ptr(n_last),
                                      ptr(dL_dimages), capacity, C.byref(grads), ptr(ws), ws.numel(),
                                      stream_handle(stream)))


def potr_selftest_wait_timeout(ws, spin_limit: int, status, stream=None):
    _check("potr_selftest_wait_timeout", lib().potr_selftest_wait_timeout(ptr(ws), ws.numel(), spin_limit,
                                                                          ptr(status), stream_handle(stream)))


def potr_prune_workspace_size(n: int) -> int:
    return int(lib().potr_prune_workspace_size(n))


def potr_prune_select(n: int, dmse, importance, alive, dmse_max: float, a: float, remaining: int, removed, ws,
                      stream=None):
    _check("potr_prune_select", lib().potr_prune_select(n, ptr(dmse), ptr(importance), ptr(alive), float(dmse_max),
                                                        float(a), int(remaining), ptr(removed), ptr(ws), ws.numel(),
                                                        stream_handle(stream)))


def potr_prune_apply(n: int, alive, opacity_logits, stream=None):
    _check("potr_prune_apply", lib().potr_prune_apply(n, ptr(alive), ptr(opacity_logits), stream_handle(stream)))


def potr_sh_compact(scene: Scene, frame: Frame, imp_view, lam: float, alpha: float, sf: float, sh_out=None,
                    sh_ycocg=None, kept=None, stream=None):
    _check("potr_sh_compact", lib().potr_sh_compact(C.byref(scene), C.byref(frame), ptr(imp_view), float(lam),
                                                    float(alpha), float(sf), ptr(sh_out), ptr(sh_ycocg), ptr(kept),
                                                    stream_handle(stream)))


def grads_struct(d: dict) -> SceneGrads:
    """SceneGrads view of a dict of parameter-shaped device tensors."""
    return SceneGrads(d["means"].data_ptr(), d["log_scales"].data_ptr(), d["quats"].data_ptr(),
                      d["opacity_logits"].data_ptr(), d["sh"].data_ptr())


def potr_adam_step(params: dict, grads: dict, m: dict, v: dict, n: int, step: int, lr, beta1=0.9, beta2=0.999,
                   eps=1e-15, stream=None):
    lrs = (C.c_float * 6)(*[float(x) for x in lr])
    _check("potr_adam_step", lib().potr_adam_step(C.byref(grads_struct(params)), C.byref(grads_struct(grads)),
                                                  C.byref(grads_struct(m)), C.byref(grads_struct(v)), n, int(step),
                                                  lrs, float(beta1), float(beta2), float(eps), stream_handle(stream)))


def potr_adam_schedule(first_step: int, count: int, lr, beta1=0.9, beta2=0.999):
    """Host table [count][7] (float32) of the per-step factors."""
    import numpy as np

    out = np.zeros((int(count), 7), np.float32)
    lrs = (C.c_float * 6)(*[float(x) for x in lr])
    _check("potr_adam_schedule", lib().potr_adam_schedule(int(first_step), int(count), lrs, float(beta1),
                                                          float(beta2), out.ctypes.data))
    return out


def potr_adam_step_scheduled(params: dict, grads: dict, m: dict, v: dict, n: int, sched, n_sched: int, step_counter,
                             beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    _check("potr_adam_step_scheduled",
           lib().potr_adam_step_scheduled(C.byref(grads_struct(params)), C.byref(grads_struct(grads)),
                                          C.byref(grads_struct(m)), C.byref(grads_struct(v)), n, ptr(sched),
                                          int(n_sched), ptr(step_counter), float(beta1), float(beta2), float(eps),
                                          stream_handle(stream)))


def potr_codec_workspace_size(n: int) -> int:
    return int(lib().potr_codec_workspace_size(n))


def potr_codec_encode(scene: Scene, eyes, n_eyes: int, params: CodecParams, nodes, n_nodes, dups, n_dups, order,
                      attrs, cube, status, ws, stream=None):
    _check("potr_codec_encode", lib().potr_codec_encode(C.byref(scene), ptr(eyes), int(n_eyes), C.byref(params),
                                                        ptr(nodes), ptr(n_nodes), ptr(dups), ptr(n_dups), ptr(order),
                                                        ptr(attrs), ptr(cube), ptr(status), ptr(ws), ws.numel(),
                                                        stream_handle(stream)))


def potr_codec_decode_workspace_size(n_nodes: int, n: int) -> int:
    return int(lib().potr_codec_decode_workspace_size(n_nodes, n))


def potr_codec_decode(nodes, n_nodes: int, dups, n_dups: int, attrs, n: int, cube, params: CodecParams, out: dict,
                      status, ws, stream=None):
    """cube: four host floats (corner x, y, z, edge); out: dict of scene-shaped device tensors."""
    cb = (C.c_double * 4)(*[float(x) for x in cube])
    _check("potr_codec_decode", lib().potr_codec_decode(ptr(nodes), int(n_nodes), ptr(dups), int(n_dups), ptr(attrs),
                                                        int(n), cb, C.byref(params), C.byref(grads_struct(out)),
                                                        ptr(status), ptr(ws), ws.numel(), stream_handle(stream)))


def potr_time_next_tile_kernel(start, stop):
    """Arm two torch.cuda.Event objects (enable_timing=True) around the next tile-pass kernel this
    thread launches (render, removal effect or backward); None, None disarms."""
    h = (lambda e: None if e is None else int(e.cuda_event))
    if start is not None:
        start.record()  # creates the events lazily; the library re-records them on the launch stream
        stop.record()
    _check("potr_time_next_tile_kernel", lib().potr_time_next_tile_kernel(h(start), h(stop)))
