"""HostPipeline: overlapped host transfers give the results of plain in-order steps."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_overlapped_steps_return_each_steps_results():
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.pipeline import HostPipeline, RemovalEffectFrame, scene_to_device

    build.build()
    sc = synth.uniform_cube_scene(5000, 61)
    cams = synth.ring_cameras(3, 3.0, 0.2, (128, 96))
    rec = synth.cameras_to_array(cams)
    scene = scene_to_device(sc)
    fr = RemovalEffectFrame(scene, rec, tile_w=16, tile_h=16, batch=256)
    fr.plan(1.5)
    rng = np.random.default_rng(0)
    # three steps with different inputs: perturbed opacities and targets
    inputs = []
    for s in range(3):
        hs = {k: t.cpu().clone() for k, t in scene.items()}
        hs["opacity_logits"] += torch.from_numpy(rng.normal(0, 0.3, sc.n).astype(np.float32))
        ht = torch.from_numpy(rng.uniform(0, 1, 3 * fr.total_pixels).astype(np.float32))
        inputs.append(({k: v.pin_memory() for k, v in hs.items()}, ht.pin_memory()))
    want = []
    for hs, ht in inputs:  # plain, one step after another
        fr.bind_scene({k: v.cuda() for k, v in hs.items()})
        d = torch.zeros(sc.n, dtype=torch.float64, device="cuda")
        i = torch.zeros_like(d)
        fr.step(ht.cuda(), d, i)
        want.append((d.cpu().numpy(), i.cpu().numpy()))
    hp = HostPipeline(fr)
    outs = [(torch.empty(sc.n, dtype=torch.float64).pin_memory(), torch.empty(sc.n, dtype=torch.float64).pin_memory())
            for _ in inputs]
    hp.upload(*inputs[0])
    for s in range(3):
        if s + 1 < 3:
            hp.upload(*inputs[s + 1])
        hp.step(*outs[s])
    hp.finish()
    for (d, i), (wd, wi) in zip(outs, want):
        assert np.array_equal(d.numpy(), wd) and np.array_equal(i.numpy(), wi)
