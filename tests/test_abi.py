"""The C-ABI library loads without a GPU, exports every entry point include/potr.h declares and
rejects null arguments on the host; without the library every call fails loudly."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "potr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(potr_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpotr():
    from paper_2601_14821_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("potr_preprocess", "potr_bin_sort", "potr_render", "potr_removal_effect"):
        assert required in names


def test_every_declared_symbol_is_exported(libpotr):
    for name in declared_functions():
        assert hasattr(libpotr, name), name


def test_binding_covers_every_symbol():
    from paper_2601_14821_gb300 import _binding

    assert set(declared_functions()) <= set(_binding.SIGNATURES)


def test_host_only_layout_and_status_strings(libpotr):
    import numpy as np

    import synth
    from paper_2601_14821_gb300 import _binding as B

    assert B.status_string(B.POTR_ERR_CAPACITY) == "tile-instance capacity exceeded"
    cams = [synth.look_at_camera((0, 0, -3), 100, 75), synth.look_at_camera((0, 0, -3), 1920, 1080)]
    info, tt, tp = B.potr_view_layout(synth.cameras_to_array(cams), B.make_config())
    rec = info.view(np.int32).reshape(2, 8)
    assert tuple(rec[0, :4]) == (100, 75, 7, 5)
    assert tuple(rec[1, :4]) == (1920, 1080, 120, 68)
    assert tt == 35 + 120 * 68 and tp == 7500 + 1920 * 1080
    with pytest.raises(B.PotrError):
        B.potr_view_layout(synth.cameras_to_array(cams), B.make_config(tile_w=16, tile_h=8))
    ws = B.potr_bin_sort_workspace_size(1000, 2, tt, 100_000)
    assert ws >= 8 * 100_000 + 16 * 2000


def test_every_entry_point_rejects_null_arguments_on_the_host(libpotr):
    """Every call that returns a status, given null pointers and zero sizes, answers
    POTR_ERR_INVALID_ARGUMENT from its host-side checks, before any device work (only null
    pointers are passed, so nothing could be launched on a device even if a check were missing)."""
    import ctypes as C

    from paper_2601_14821_gb300 import _binding as B

    floats = (C.c_float, C.c_double)
    checked = []
    for name, (res, args) in sorted(B.SIGNATURES.items()):
        if res is not B._I32 or name in ("potr_version", "potr_time_next_tile_kernel"):
            continue  # (NULL, NULL) is the hook's documented disarm, tested below
        vals = [0.0 if a in floats else (None if a is B._P or issubclass(a, C._Pointer) else 0) for a in args]
        assert getattr(B.lib(), name)(*vals) == B.POTR_ERR_INVALID_ARGUMENT, name
        checked.append(name)
    for required in ("potr_preprocess", "potr_bin_sort", "potr_render", "potr_removal_effect",
                     "potr_render_backward", "potr_sh_compact", "potr_codec_encode", "potr_codec_decode"):
        assert required in checked


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libpotr.so every call raises at once (there is no CPU fallback to take over)."""
    import numpy as np

    from paper_2601_14821_gb300 import _binding as B

    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "libpotr.so"))
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()
    with pytest.raises(RuntimeError, match="not built"):
        B.potr_view_layout(np.zeros((1, 18), np.float32), B.make_config())


def test_timing_hook_and_status_word_on_the_host(libpotr):
    """The tile-kernel timing hook takes both events or neither; the device status word has the
    layout the header gives (code, non-finite splat count, required instances) and the
    non-finite code its string."""
    import ctypes as C

    from paper_2601_14821_gb300 import _binding as B

    L = B.lib()
    assert L.potr_time_next_tile_kernel(None, None) == B.POTR_OK
    assert L.potr_time_next_tile_kernel(C.c_void_p(16), None) == B.POTR_ERR_INVALID_ARGUMENT
    assert L.potr_time_next_tile_kernel(None, C.c_void_p(16)) == B.POTR_ERR_INVALID_ARGUMENT
    assert B.DeviceStatus.code.offset == 0 and B.DeviceStatus.n_nonfinite.offset == 4
    assert B.DeviceStatus.required_instances.offset == 8 and C.sizeof(B.DeviceStatus) == 16
    assert B.status_string(B.POTR_ERR_NUMERIC) == "non-finite input"


def test_static_sort_limits_fit_its_scratch(libpotr):
    """Every call within potr_bin_sort_static's advertised limits fits its 56 MiB scratch: the
    workspace of the largest instance count and (view, splat) count, split over 1 to 64 views."""
    from paper_2601_14821_gb300 import _binding as B

    cap, vs = int(B.POTR_STATIC_MAX_INSTANCES), int(B.POTR_STATIC_MAX_VIEW_SPLATS)
    for views in (1, 2, 4, 16, 64):
        need = B.potr_bin_sort_workspace_size(vs // views, views, 1 << 20, cap)
        assert 0 < need <= 56 << 20, (views, need)


def test_workspace_sizes_of_the_removal_and_backward_passes(libpotr):
    """The documented workspace formulas (host only): the removal pass keeps 16 bytes of block
    sums per instance (32 with importance) and 20 bytes per tile, the backward pass 36 bytes of
    partials per instance and 52 bytes per (view, splat); both are 0 for non-positive sizes and
    grow with every argument."""
    from paper_2601_14821_gb300 import _binding as B

    cap, tiles, vk = 1_000_000, 3600, 500_000
    r0 = B.potr_removal_workspace_size(cap, tiles, False)
    r1 = B.potr_removal_workspace_size(cap, tiles, True)
    assert 16 * cap + 20 * tiles <= r0 < 16 * cap + 20 * tiles + 4 * 256
    assert 32 * cap + 20 * tiles <= r1 < 32 * cap + 20 * tiles + 4 * 256
    assert B.potr_removal_workspace_size(cap + 1000, tiles, True) > r1
    assert B.potr_removal_workspace_size(cap, tiles + 1000, True) > r1
    assert B.potr_removal_workspace_size(0, tiles, True) == 0 and B.potr_removal_workspace_size(cap, 0, True) == 0
    b = B.potr_render_backward_workspace_size(cap, vk)
    assert b == 36 * cap + 52 * vk
    assert B.potr_render_backward_workspace_size(0, vk) == 0 and B.potr_render_backward_workspace_size(cap, 0) == 0


def test_preprocess_rejects_tile_shapes_other_than_256_pixels(libpotr):
    """The projection divides by the tile size as a product with its reciprocal, exact only for
    the power-of-two sizes that tile_w tile_h = 256 allows: any other shape is refused on the
    host.  The structs hold host addresses, so this runs only where no GPU is visible."""
    import ctypes as C

    import torch

    from paper_2601_14821_gb300 import _binding as B

    if torch.cuda.is_available():
        pytest.skip("host-only check")
    buf = (C.c_float * 64)()
    addr = C.cast(buf, C.c_void_p).value
    scene = B.Scene(addr, addr, addr, addr, addr, 1)
    frame = B.Frame(addr, addr, 1, 1, 1)
    views = B.Views(*([addr] * len(B.Views._fields_)))
    for tw, th in ((12, 12), (16, 8), (0, 256), (-16, -16)):
        cfg = B.make_config(tile_w=tw, tile_h=th)
        st = B.lib().potr_preprocess(C.byref(scene), C.byref(frame), C.byref(cfg), C.byref(views), None, None)
        assert st == B.POTR_ERR_INVALID_ARGUMENT, (tw, th)
