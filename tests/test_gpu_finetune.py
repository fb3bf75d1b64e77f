"""Fine-tuning (Section IV-F) on the device: the fused Adam step against the Adam oracle, and
the loop lowering the photometric loss of a perturbed scene."""
import numpy as np
import pytest

import synth
from oracle import adam as oadam

pytestmark = pytest.mark.gpu

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def test_adam_step_matches_oracle():
    import torch

    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300 import build

    build.build()
    rng = np.random.default_rng(3)
    n = 4099
    shapes = {"means": (3, n), "log_scales": (3, n), "quats": (4, n), "opacity_logits": (n,), "sh": (16, 3, n)}
    p = {k: rng.normal(size=s).astype(np.float32) for k, s in shapes.items()}
    p["opacity_logits"][:7] = -np.inf  # pruned splats
    lr = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)
    dev = {k: torch.from_numpy(a.copy()).cuda() for k, a in p.items()}
    m = {k: torch.zeros_like(t) for k, t in dev.items()}
    v = {k: torch.zeros_like(t) for k, t in dev.items()}
    op = {k: a.astype(np.float64) for k, a in p.items()}
    om = {k: np.zeros_like(a) for k, a in op.items()}
    ov = {k: np.zeros_like(a) for k, a in op.items()}
    for t in range(1, 6):
        g = {k: (rng.normal(size=s) * 10.0 ** rng.uniform(-4, 1)).astype(np.float32) for k, s in shapes.items()}
        g["opacity_logits"][:7] = 0.0
        g["sh"][5] = 0.0  # a plane with no gradient yet
        gd = {k: torch.from_numpy(a).cuda() for k, a in g.items()}
        B.potr_adam_step(dev, gd, m, v, n, t, lr)
        og = oadam.split_groups({k: a.astype(np.float64) for k, a in g.items()})
        for name, lr_i in zip(oadam.GROUPS, lr):
            pg, mg, vg = (oadam.split_groups(x)[name] for x in (op, om, ov))
            oadam.step(pg, og[name], mg, vg, t, lr_i)
        torch.cuda.synchronize()
        for k in KEYS:
            got = dev[k].cpu().numpy().astype(np.float64)
            fin = np.isfinite(op[k])
            np.testing.assert_allclose(got[fin], op[k][fin], rtol=2e-6, atol=1e-6, err_msg=f"{k} step {t}")
            assert np.array_equal(np.isfinite(got), fin)


def test_finetune_lowers_the_loss_of_a_perturbed_scene():
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.finetune import FineTuner
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    build.build()
    sc = synth.uniform_cube_scene(4000, 23)
    cams = synth.ring_cameras(6, 3.0, 0.3, (128, 96))
    rec = synth.cameras_to_array(cams)
    cfg = dict(tile_w=16, tile_h=16, batch=256)
    ref = scene_to_device(sc)
    targets = []
    for v in range(len(cams)):
        f = RemovalEffectFrame(ref, rec[v:v + 1], with_importance=False, **cfg)
        f.plan()
        img = f.image_buffer()
        f.render(img)
        targets.append(img)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    pert = {k: t.clone() for k, t in ref.items()}
    pert["sh"][0] += torch.from_numpy(rng.normal(0, 0.3, (3, sc.n)).astype(np.float32)).cuda()
    pert["means"] += torch.from_numpy(rng.normal(0, 0.003, (3, sc.n)).astype(np.float32)).cuda()
    ft = FineTuner(pert, rec, targets, lam=0.2, extent=3.0, **cfg)
    first = ft.run(len(cams), order=list(range(len(cams))))
    losses = []
    for _ in range(5):
        ft.run(60, seed=len(losses))
        tot = 0.0
        for v in range(len(cams)):  # loss over every view, without stepping
            fr = ft.frames[v]
            img, tf, nl, dL = ft._buffers(fr)
            fr.preprocess()
            fr.bin_sort()
            fr.render(img)
            ft.loss.zero_()
            fr.loss_grad(img, targets[v], 0.2, dL, ft.loss)
            tot += float(ft.loss.item())
        losses.append(tot / len(cams))
    assert losses[-1] < 0.5 * first and losses[-1] < losses[0]
    assert all(torch.isfinite(t).all() for t in pert.values())


def test_scheduled_adam_equals_host_step_adam():
    """Adam with t from the device counter and the host-made factor table gives the bits of
    Adam with t passed from the host, step after step; steps past the table change nothing."""
    import torch

    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300 import build

    build.build()
    rng = np.random.default_rng(8)
    n = 3001
    shapes = {"means": (3, n), "log_scales": (3, n), "quats": (4, n), "opacity_logits": (n,), "sh": (16, 3, n)}
    lr = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)
    p0 = {k: rng.normal(size=s).astype(np.float32) for k, s in shapes.items()}
    a = {k: torch.from_numpy(x.copy()).cuda() for k, x in p0.items()}
    b = {k: torch.from_numpy(x.copy()).cuda() for k, x in p0.items()}
    ma, va = ({k: torch.zeros_like(t) for k, t in a.items()} for _ in range(2))
    mb, vb = ({k: torch.zeros_like(t) for k, t in b.items()} for _ in range(2))
    rows = 4
    sched = torch.from_numpy(B.potr_adam_schedule(1, rows, lr).reshape(-1)).cuda()
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    for t in range(1, rows + 1):
        g = {k: torch.from_numpy(rng.normal(size=s).astype(np.float32)).cuda() for k, s in shapes.items()}
        B.potr_adam_step(a, g, ma, va, n, t, lr)
        B.potr_adam_step_scheduled(b, g, mb, vb, n, sched, rows, counter)
        torch.cuda.synchronize()
        for k in KEYS:
            assert torch.equal(a[k], b[k]) and torch.equal(ma[k], mb[k]) and torch.equal(va[k], vb[k]), (k, t)
    before = {k: t.clone() for k, t in b.items()}
    B.potr_adam_step_scheduled(b, g, mb, vb, n, sched, rows, counter)  # step 5: past the table
    torch.cuda.synchronize()
    assert int(counter.item()) == rows + 1
    assert all(torch.equal(before[k], b[k]) for k in KEYS)


def test_finetune_graph_replay_equals_eager_steps():
    """The fine-tuner with each view's iteration captured in a CUDA graph ends with the same
    parameter bits as issuing the same iterations eagerly."""
    import torch

    from paper_2601_14821_gb300 import build
    from paper_2601_14821_gb300.finetune import FineTuner
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    build.build()
    sc = synth.uniform_cube_scene(3000, 31)
    cams = synth.ring_cameras(3, 3.0, 0.3, (96, 64))
    rec = synth.cameras_to_array(cams)
    cfg = dict(tile_w=16, tile_h=16, batch=128)
    ref = scene_to_device(sc)
    targets = []
    for v in range(len(cams)):
        f = RemovalEffectFrame(ref, rec[v:v + 1], with_importance=False, **cfg)
        f.plan()
        img = f.image_buffer()
        f.render(img)
        targets.append(img.clone())
    rng = np.random.default_rng(2)
    noise = torch.from_numpy(rng.normal(0, 0.2, (3, sc.n)).astype(np.float32)).cuda()
    out = []
    for graphs in (False, True):
        params = {k: t.clone() for k, t in ref.items()}
        params["sh"][0] += noise
        ft = FineTuner(params, rec, targets, lam=0.2, extent=3.0, graphs=graphs, **cfg)
        ft.run(12, order=[0, 1, 2])
        torch.cuda.synchronize()
        out.append({k: t.cpu().numpy() for k, t in params.items()})
        if graphs:
            assert all(g is not None for g in ft._graphs)
    for k in KEYS:
        assert np.array_equal(out[0][k], out[1][k]), k
