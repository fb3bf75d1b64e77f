"""potr_bin_sort_static: the sort for callers that cannot allocate device memory.

Some callers own no allocator for the device -- a plug-in inside a host application that
manages all GPU memory, or a loop where allocating would synchronise the device.  This entry
point takes only their inputs and outputs and uses scratch held inside the library.  The test
drives it through the C ABI and checks it against potr_bin_sort (bit-exact, like every
integer output in these tests) on two calls in a row, and that oversized requests are refused.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _frame(scene, cams):
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    build.build()
    fr = RemovalEffectFrame(scene_to_device(scene), synth.cameras_to_array(cams), tile_w=16, tile_h=16, batch=256)
    fr.plan()
    torch.cuda.synchronize()
    return fr


def _sorted_outputs(fr, tiles, vals, ranges):
    m = fr.instance_count()
    return (tiles[:m].cpu().numpy().view(np.uint32), vals[:m].cpu().numpy().view(np.uint32),
            ranges.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("which", ["tiny", "mixed"])
def test_static_scratch_sort_matches_workspace_sort_twice(which):
    import torch

    from paper_2601_14821_gb300 import _binding as B

    if which == "tiny":
        w = synth.workload("tiny")
        scene, cams = w.scene, w.cameras
    else:
        scene = synth.uniform_cube_scene(5000, 77)
        cams = [synth.look_at_camera((0.0, 0.3, -3.0), 200, 150), synth.look_at_camera((2.5, -0.2, -1.5), 96, 160)]
    fr = _frame(scene, cams)
    want = _sorted_outputs(fr, fr.tiles, fr.vals, fr.ranges)
    assert want[0].size > 1000
    for call in range(2):
        tiles = torch.full_like(fr.tiles, -1)
        vals = torch.full_like(fr.vals, -1)
        ranges = torch.full_like(fr.ranges, -1)
        status = torch.zeros(2, dtype=torch.int64, device=fr.device)
        B.potr_bin_sort_static(fr.views, fr.frame, fr.cfg, fr.n, fr.capacity, tiles, vals, ranges, status)
        torch.cuda.synchronize()
        assert status.tolist() == [0, 0], call
        got = _sorted_outputs(fr, tiles, vals, ranges)
        for g, e in zip(got, want):
            assert np.array_equal(g, e), call


def _check_refused(B, fr, n, capacity):
    """A refused call enqueues nothing: the outputs keep their sentinel values."""
    import torch

    tiles = torch.full_like(fr.tiles, -7)
    vals = torch.full_like(fr.vals, -7)
    ranges = torch.full_like(fr.ranges, -7)
    status = torch.full((2,), -7, dtype=torch.int64, device=fr.device)
    with pytest.raises(B.PotrError) as e:
        B.potr_bin_sort_static(fr.views, fr.frame, fr.cfg, n, capacity, tiles, vals, ranges, status)
    assert e.value.status == B.POTR_ERR_TOO_LARGE
    torch.cuda.synchronize()
    for t in (tiles, vals, ranges, status):
        assert bool((t == -7).all())


def test_static_scratch_sort_rejects_oversize():
    """Both limits: more instances than POTR_STATIC_MAX_INSTANCES, and more (view, splat) pairs
    than POTR_STATIC_MAX_VIEW_SPLATS (a 1,048,577-splat scene in one view)."""
    from paper_2601_14821_gb300 import _binding as B

    w = synth.workload("tiny")
    fr = _frame(w.scene, w.cameras)
    _check_refused(B, fr, fr.n, B.POTR_STATIC_MAX_INSTANCES + 1)
    big = synth.uniform_cube_scene(int(B.POTR_STATIC_MAX_VIEW_SPLATS) + 1, 5)
    fr2 = _frame(big, w.cameras)
    assert fr2.n * fr2.n_views == B.POTR_STATIC_MAX_VIEW_SPLATS + 1
    _check_refused(B, fr2, fr2.n, min(fr2.capacity, int(B.POTR_STATIC_MAX_INSTANCES)))
