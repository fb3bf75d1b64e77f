"""The compression driver end to end on the tiny workload: pruning, SH compaction and encoding
chained on the device; the pruned set, the encoded scene and the bitstream are checked against
the stages' definitions and the codec oracle."""
import numpy as np
import pytest

import synth
from oracle import codec as ocodec
from oracle.sh_compact import camera_centre

pytestmark = pytest.mark.gpu

CFG = dict(tile_w=16, tile_h=16, batch=256)


def _setup():
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.pipeline import scene_to_device

    build.build()
    w = synth.workload("tiny")
    scene = scene_to_device(w.scene)
    rec = synth.cameras_to_array(w.cameras)
    be = BatchedRemovalEffect(scene, rec, **CFG)
    be.plan()
    targets = torch.empty(3 * be.total_pixels, dtype=torch.float32, device="cuda")
    be.render(targets)
    d0 = torch.zeros(w.scene.n, dtype=torch.float64, device="cuda")
    be.step(targets, d0, torch.zeros_like(d0))
    # dMSE_MAX at the median |dMSE| of the unpruned scene, so that many splats go
    dmax = float(np.median(np.abs(d0.cpu().numpy())))
    return w, scene, rec, targets, dmax


def test_compress_prunes_compacts_and_encodes():
    from paper_2601_14821_gb300.compress import compress

    w, scene, rec, targets, dmax = _setup()
    eyes = np.array([camera_centre(c) for c in w.cameras])
    before = {k: t.cpu().numpy() for k, t in scene.items()}
    out = compress(scene, rec, targets=targets, iterations=4, dmse_max_value=dmax, eyes=eyes, **CFG)
    n = w.scene.n
    keep = out["keep"].cpu().numpy()
    logits = scene["opacity_logits"].cpu().numpy()
    # the live set: finite logits exactly at keep, the removed ones at -inf, nothing else moved
    assert np.all(np.isfinite(before["opacity_logits"]))
    assert np.array_equal(np.nonzero(np.isfinite(logits))[0], keep)
    assert np.all(logits[~np.isfinite(logits)] == -np.inf)
    assert np.array_equal(logits[keep], before["opacity_logits"][keep])
    counts = out["alive_after_iteration"]
    assert len(counts) == 4 and all(a >= b for a, b in zip([n] + counts, counts))
    assert counts[-1] == keep.size and 0 < keep.size < n
    # the encoded scene: the live splats in input order, SH replaced by the compaction's
    sub = {k: t.cpu().numpy() for k, t in out["scene"].items()}
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        assert np.array_equal(sub[k], before[k][..., keep]), k
    assert sub["sh"].shape == (16, 3, keep.size) and np.all(np.isfinite(sub["sh"]))
    # the bitstream is the codec oracle's encoding of that scene, byte for byte
    sc = synth.Scene(sub["means"], sub["log_scales"], sub["quats"], sub["opacity_logits"], sub["sh"])
    want = ocodec.encode(sc, eyes, p=ocodec.params(0.5))
    assert out["raw"] == want["raw"]
    assert ocodec.decode(out["compressed"])["means"].shape == (3, keep.size)


def test_compress_with_a_fine_tuning_cycle():
    from paper_2601_14821_gb300.compress import compress

    w, scene, rec, targets, dmax = _setup()
    out = compress(scene, rec, targets=targets, iterations=2, dmse_max_value=dmax, ft_cycles=1, ft_iterations=20,
                   **CFG)
    m = int(out["keep"].numel())
    assert len(out["losses"]) == 1 and np.isfinite(out["losses"][0])
    assert out["scene"]["means"].shape[-1] == m
    assert ocodec.decode(out["compressed"])["means"].shape == (3, m)
