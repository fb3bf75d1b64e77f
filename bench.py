"""Benchmark of the removal-effect path on one GB300 (or N GPUs of one node, weak scaling).

A step is one pass of the whole path over one frame: activation + EWA projection of 1M
splats into 16 views of 1280x720, tile binning + radix sort of every (tile, splat) instance,
and the removal-effect pass with the per-splat dMSE_k / I_k reduction.  Inputs (the 236 MB of
splat parameters, the 0.77 GB of per-view raster records, 0.45 GB of instances) are larger than
the 129 MB L2, so no L2 flush is needed between steps.

Printed (one JSON line on rank 0): the device-timed throughput of the batched frame
(``value``, views/s), the same frame replayed as a CUDA graph, the one-view-per-launch form,
Gblend/s (evaluated pixel-splat pairs per second of the removal kernel), the roofline of the
removal kernel (FP32 ALU), the end-to-end number through host buffers, the clocks seen
during the timed region, and the CPU oracle timed on a bounded sample.  Beside them: the
fine-tuning forward + backward step and the Adam fine-tuning loop (``fwd_bwd``), the whole
iterative pruning of the scene with the SH energy compaction and the encoder of the pruned
scene (``pruning``), the 200 views of mixed resolution as one frame against one view per launch
(``multiview``), and the 6M-splat, 300-view 1080p workload in 8-view chunks with its fine-tuning
step (``large``; skipped with ``--no-large``).  ``rooflines`` holds the FP32 roofline of each tile
kernel (compositing, removal effect, backward), each kernel timed alone with CUDA events.

``--impl reference`` times the CPU oracle itself on the same workload (all views per step, every
host core).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "removal-effect views/s & Gblend/s (batched vs per-view); fwd+bwd ms/step"
WORKLOAD = "scene"
CFG = dict(tile_w=16, tile_h=16, batch=128)
# Algorithmic FP32 work (FMA = 2 FLOP), counted from the operation spec of the method's per-pixel
# walks in the roofline's unit, the evaluated (pixel, list position) pair -- front to back up to
# the pixel's termination, back to front over the positions below its n_last: every evaluated
# pair takes its exponent, exp2 (its FMA count) and alpha; compositing and the removal or
# backward terms are counted where the pixel composites the splat.  The kernels skip exp2 where a
# log-domain comparison already decides alpha < alpha_min; `frac_strict` counts exp2 and alpha
# only where they are evaluated, for comparison.
FLOP_EXPONENT = 9        # dx, dy, A dx^2 + B dx dy + C dy^2 (per evaluated pair)
FLOP_ALPHA = 17          # exp2 (3 add + 6 FMA), o * G, min (per evaluated pair)
FLOP_COMPOSITE = 9       # T (1 - alpha), w = alpha T, three colour FMAs (composited pairs)
FLOP_REMOVAL = 26        # T recovery, ratio, PD and dSE over 3 channels, suffix update (composited pairs)
FLOP_BWD = 45            # backward, per composited pair: T recovery, dL/dalpha from the suffix, the nine
                         # per-pair gradients (centre, A, B, C, opacity, colour), suffix update
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
PEAK_FP32_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
# DRAM bytes (read + written) per launch and view of each tile kernel, from ncu captures of the
# kernel as it is built now (None: no capture of the current kernel yet).
# removal: 622.3 + 168.0 MB over 4 views; render: 123.0 + 22.9 MB over 4 views (scene workload).
# The backward tile kernel has changed (six CTAs per SM) since its capture (945.9 + 158.1 MB over
# 8 views at five), so it reports none.
DRAM_BYTES_PER_VIEW = {"removal_kernel": 790.3e6 / 4, "render_kernel": 145.9e6 / 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--views", type=int, default=0, help="use only the first V views (profiling cases)")
    ap.add_argument("--only-batched", action="store_true", help="time the batched frame only (profiling cases)")
    ap.add_argument("--only-fwdbwd", action="store_true", help="time the fine-tuning step only (profiling case)")
    ap.add_argument("--only-pruning", action="store_true",
                    help="run the pruning, SH compaction, codec and POTR-FT section only (profiling case)")
    ap.add_argument("--no-large", action="store_true", help="skip the 6M-splat, 300-view 1920x1080 workload")
    ap.add_argument("--no-multiview", action="store_true", help="skip the 3M-splat, 200-view workload")
    ap.add_argument("--profile-timed", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# workload construction
# ------------------------------------------------------------------------------------------

def make_targets_gpu(w, frame_cls, scene_to_device, cams_rec, torch):
    """Workload recipe: render of the scene with a seeded 5 % of the splats dropped, plus
    N(0, 0.01) noise per view (input preparation, outside the timed region)."""
    import synth

    keep = synth.target_drop_mask(w.scene.n, w.target_drop, w.seed)
    tf = frame_cls(scene_to_device(w.scene.subset(keep)), cams_rec, with_importance=False, **CFG)
    tf.plan()
    img = tf.image_buffer()
    tf.render(img)
    torch.cuda.synchronize()
    noise = np.concatenate([synth.target_noise((3, c.height, c.width), w.target_noise, w.seed, v).reshape(-1)
                            for v, c in enumerate(w.cameras)])
    img += torch.from_numpy(noise).to(img.device)
    del tf
    return img


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_targets(w, views, cores: int) -> list:
    """The workload's targets for the given views from the oracle (render of the scene with the
    seeded 5 % dropped, plus noise), views in parallel (input preparation, not timed)."""
    import concurrent.futures as cf

    import oracle
    import synth

    ocfg = oracle.make_config(tile_w=CFG["tile_w"], tile_h=CFG["tile_h"])
    sc2 = w.scene.subset(synth.target_drop_mask(w.scene.n, w.target_drop, w.seed))
    act = oracle.activate(sc2)

    def one(v):
        tv = oracle.prepare_view(sc2, w.cameras[v], ocfg, act)
        img, *_ = oracle.render(tv, tv["vals"], tv["ranges"], w.cameras[v], ocfg)
        return (img + synth.target_noise(img.shape, w.target_noise, w.seed, v)).astype(np.float32)

    oracle.set_threads(1)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(cores, len(views)))) as ex:
        return list(ex.map(one, views))


def oracle_frame_seconds(w, views, targets, cores: int) -> float:
    """The CPU oracle on whole views of the workload -- activation, then per view projection,
    binning + stable sort and the removal effect with importance, the views' dMSE_k / I_k added in
    view order -- on ``cores`` host threads: the views run concurrently (the oracle's C code runs
    outside the interpreter lock), each view's tiles on cores // views threads when there are
    more cores than views.  Returns the wall seconds."""
    import concurrent.futures as cf

    import oracle

    ocfg = oracle.make_config(tile_w=CFG["tile_w"], tile_h=CFG["tile_h"])
    workers = max(1, min(cores, len(views)))
    oracle.set_threads(max(1, cores // workers))
    t0 = time.perf_counter()
    act = oracle.activate(w.scene)

    def one(i):
        cam = w.cameras[views[i]]
        pv = oracle.prepare_view(w.scene, cam, ocfg, act)
        return oracle.removal_effect(pv, pv["vals"], pv["ranges"], cam, ocfg, targets[i])

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        parts = list(ex.map(one, range(len(views))))
    dmse = np.zeros(w.scene.n)
    imp = np.zeros(w.scene.n)
    for i, (d, im) in enumerate(parts):
        P = float(w.cameras[views[i]].pixels)
        dmse += d / (3.0 * P) / len(views)
        imp += im / P / len(views)
    secs = time.perf_counter() - t0
    oracle.set_threads(1)
    return secs


def tile_kernel_ms(B, torch, fn, reps: int) -> float:
    """Mean device time of the tile-pass kernel launched by ``fn`` (render, removal effect or
    backward), measured with CUDA events the library records on the launch stream around that
    kernel alone (potr_time_next_tile_kernel)."""
    evs = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        B.potr_time_next_tile_kernel(a, b)
        fn()
        evs.append((a, b))
    B.potr_time_next_tile_kernel(None, None)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def render_flops(pc: dict, strict: bool = False) -> float:
    alpha_pairs = pc["passed"] if strict else pc["examined"]
    return FLOP_EXPONENT * pc["examined"] + FLOP_ALPHA * alpha_pairs + FLOP_COMPOSITE * pc["composited"]


def removal_flops(pc: dict, strict: bool = False) -> float:
    walked = pc["examined"] + pc["back_positions"]
    alpha_pairs = pc["passed"] + pc["back_passed"] if strict else walked
    return FLOP_EXPONENT * walked + FLOP_ALPHA * alpha_pairs + (FLOP_COMPOSITE + FLOP_REMOVAL) * pc["composited"]


def bwd_flops(pc: dict, strict: bool = False) -> float:
    alpha_pairs = pc["back_passed"] if strict else pc["back_positions"]
    return FLOP_EXPONENT * pc["back_positions"] + FLOP_ALPHA * alpha_pairs + FLOP_BWD * pc["composited"]


def roofline_entry(kernel: str, flops: float, ms: float, views: int, workload: str,
                   flops_strict: float | None = None) -> dict:
    achieved = flops / (ms / 1e3) / 1e12
    # the captures were made on the scene (tile kernels) and grad (backward) workloads; other
    # workloads (other resolutions and densities) get no traffic figure
    per_view = DRAM_BYTES_PER_VIEW.get(kernel) if workload in ("scene", "grad") else None
    return {"kernel": kernel, "workload": workload, "bound": "alu", "achieved": achieved,
            "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s", "frac": achieved / PEAK_FP32_TFLOPS,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (unit counts and maximum clock)",
            "traffic": None if per_view is None else per_view * views, "flops_per_launch": flops,
            "kernel_ms": ms,
            "frac_strict": None if flops_strict is None else flops_strict / (ms / 1e3) / 1e12 / PEAK_FP32_TFLOPS}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

def run_ours(args):
    import torch

    import synth
    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300 import build as potr_build
    from paper_2601_14821_gb300 import dist as D
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    rank, local, world = D.env_ranks()
    potr_build.build()
    torch.cuda.set_device(local)
    D.init("nccl")
    dev = torch.device("cuda", local)
    if args.only_fwdbwd:
        out = fwd_bwd_step_ms(args, dev, D)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "fwd_bwd": out, "profiling_case": True}))
        return
    if args.only_pruning:
        out = prune_run(args, dev, D)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "pruning": out, "profiling_case": True}))
        return
    w = synth.workload(WORKLOAD)
    if args.views:
        w.cameras = w.cameras[: args.views]
    n_views = len(w.cameras)
    cams_rec = synth.cameras_to_array(w.cameras)
    scene_d = scene_to_device(w.scene, dev)
    frame = RemovalEffectFrame(scene_d, cams_rec, device=dev, **CFG)
    n_inst = frame.plan()
    targets = make_targets_gpu(w, RemovalEffectFrame, scene_to_device, cams_rec, torch)
    dmse = torch.zeros(frame.n, dtype=torch.float64, device=dev)
    imp = torch.zeros(frame.n, dtype=torch.float64, device=dev)

    def step():
        frame.preprocess()
        frame.bin_sort()
        frame.removal_effect(targets, dmse, imp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps of the batched frame, per-stage events on the launch stream
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid else None)
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    D.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = B.potr_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if args.profile_timed:
        torch.cuda.profiler.start()
    t_start.record()
    for i in range(K):
        ev[i][0].record()
        frame.preprocess()
        ev[i][1].record()
        frame.bin_sort()
        ev[i][2].record()
        frame.removal_effect(targets, dmse, imp)
        ev[i][3].record()
    t_end.record()
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.profiler.stop()
    D.barrier()
    launches = B.potr_launch_count() - l0
    clk = clocks.stop()
    ms_total = D.max_over_ranks(t_start.elapsed_time(t_end), dev)
    stage = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in ev])
    stage_ms = stage.mean(axis=0)
    ms_step = ms_total / K
    value = world * n_views * K / (ms_total / 1e3)

    if args.only_batched:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "views/s", "views": n_views,
                              "stage_ms": {"preprocess": stage_ms[0], "bin_sort": stage_ms[1],
                                           "removal_effect": stage_ms[2]}, "instances": int(n_inst),
                              "gpu_launches": int(launches), "profiling_case": True}))
        return

    # ---- CUDA graph of one whole step, replayed
    graph_vps = None
    try:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            step()
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(K):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        graph_vps = world * n_views * K / (D.max_over_ranks(a.elapsed_time(b), dev) / 1e3)
        del g
    except Exception as exc:  # reported, not hidden
        graph_vps = f"capture failed: {exc}"

    # ---- one view per launch chain
    per_frames = [RemovalEffectFrame(scene_d, cams_rec[v:v + 1], device=dev, **CFG) for v in range(n_views)]
    for f in per_frames:
        f.plan()
    tviews = [targets[3 * int(frame.info_np[v]["pixel_base"]): 3 * int(frame.info_np[v]["pixel_base"])
                      + 3 * w.cameras[v].pixels] for v in range(n_views)]

    def per_view_step():
        for f, t in zip(per_frames, tviews):
            f.step(t, dmse, imp, n_views_total=n_views)

    for _ in range(args.warmup):
        per_view_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(K):
        per_view_step()
    b.record()
    torch.cuda.synchronize()
    per_view_vps = world * n_views * K / (D.max_over_ranks(a.elapsed_time(b), dev) / 1e3)
    del per_frames

    # ---- exact pair counts -> Gblend/s and the ALU rooflines of the tile kernels, each timed
    # alone (events recorded by the library around the kernel on its launch stream)
    pc = frame.pair_stats()
    torch.cuda.synchronize()
    pairs = pc["examined"] + pc["back_positions"]
    flops = removal_flops(pc)
    t_removal = stage_ms[2] / 1e3
    gblend = world * pairs / t_removal / 1e9
    ms_removal_kernel = tile_kernel_ms(B, torch, lambda: frame.removal_effect(targets, dmse, imp), K)
    img_buf = frame.image_buffer()
    ms_render_kernel = tile_kernel_ms(B, torch, lambda: frame.render(img_buf), K)
    flops_render = render_flops(pc)
    rl_removal = roofline_entry("removal_kernel", flops, ms_removal_kernel, n_views, "scene",
                                removal_flops(pc, strict=True))
    rl_render = roofline_entry("render_kernel", flops_render, ms_render_kernel, n_views, "scene",
                               render_flops(pc, strict=True))
    del img_buf

    # ---- end to end through host buffers (pinned): parameters + targets in, dMSE + I out
    host_scene = {k: v.cpu().pin_memory() for k, v in scene_d.items()}
    host_targets = targets.cpu().pin_memory()
    host_dmse = torch.empty_like(dmse, device="cpu").pin_memory()
    host_imp = torch.empty_like(imp, device="cpu").pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host_scene.values()) + host_targets.numel() * 4
    d2h = 2 * dmse.numel() * 8

    from paper_2601_14821_gb300.pipeline import HostPipeline

    hp = HostPipeline(frame)

    def e2e_run(steps):
        hp.copy.wait_stream(torch.cuda.current_stream(dev))  # copies start inside the timed region
        hp.upload(host_scene, host_targets)
        for i in range(steps):
            if i + 1 < steps:
                hp.upload(host_scene, host_targets)  # the next step's inputs, during this step
            hp.step(host_dmse, host_imp)

    e2e_run(args.warmup)
    hp.finish()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    D.barrier()
    a.record()
    e2e_run(K)
    hp.join()  # the last results are on the host when the compute stream passes this point
    b.record()
    torch.cuda.synchronize()
    e2e_vps = world * n_views * K / (D.max_over_ranks(a.elapsed_time(b), dev) / 1e3)

    # ---- fine-tuning step: 1M splats, 8 views 1280x720, L1 + squared-error loss (lambda 0.2)
    fwd_bwd = fwd_bwd_step_ms(args, dev, D)

    # ---- iterative pruning (Section IV-C): 48 iterations over the 16 views of the scene
    pruning = prune_run(args, dev, D)

    # ---- many views of uneven resolution: all 200 views as one frame (one launch per stage),
    # against the one-view-per-launch form; the 6M-splat, 300-view 1080p workload in view chunks
    multiview = None if args.no_multiview else multiview_config(args, dev, D, "batched", None, per_view=True)
    large = None if args.no_large else multiview_config(args, dev, D, "large", 8, fwd_bwd=True)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        views = list(range(n_views))
        tg_cpu = oracle_targets(w, views, cores)
        secs = oracle_frame_seconds(w, views, tg_cpu, cores)
        cpu = {"value": len(views) / secs, "unit": "views/s", "cores": cores, "kind": "oracle",
               "sample": f"all {len(views)} views of the workload ({secs:.1f} s on {cores} host threads: views "
                         "concurrently, activation, projection, binning + stable sort, removal effect and "
                         "importance, dMSE_k / I_k added in view order)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": scene_config(int(frame.n), n_views, world),
            "form": "batched frame (all views in one launch per stage)", "instances": int(n_inst),
            "stage_ms": {"preprocess": stage_ms[0], "bin_sort": stage_ms[1], "removal_effect": stage_ms[2]},
            "graph_views_per_s": graph_vps,
            "per_view_views_per_s": per_view_vps,
            "gblend_per_s": gblend,
            "pairs": pc,
            "fwd_bwd_ms_per_step": fwd_bwd["store"],
            "fwd_bwd": fwd_bwd,
            "pruning": pruning,
            "multiview": multiview,
            "large": large,
            "roofline": rl_removal,
            "rooflines": [rl_removal, rl_render] + ([fwd_bwd["roofline"]] if fwd_bwd.get("roofline") else []),
            "removal_stage_tflops": flops / t_removal / 1e12,
            "e2e": {"value": e2e_vps, "unit": "views/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))


def fwd_bwd_step_ms(args, dev, D) -> dict:
    """One fine-tuning forward + backward step on the gradient workload (1M splats, 8 views
    1280x720): preprocess, bin + sort, render, loss and dL/dc, backward rasterizer and the
    per-splat parameter adjoint.  Timed with the final transmittance stored by the forward
    pass and with it recomputed inside the backward kernel."""
    import torch

    import synth
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    w = synth.workload("grad")
    cams_rec = synth.cameras_to_array(w.cameras)
    scene_d = scene_to_device(w.scene, dev)
    fr = RemovalEffectFrame(scene_d, cams_rec, device=dev, with_importance=False, **CFG)
    fr.plan()
    img = fr.image_buffer()
    fr.render(img)
    torch.cuda.synchronize()
    noise = np.concatenate([synth.target_noise((3, c.height, c.width), w.target_noise, w.seed, v).reshape(-1)
                            for v, c in enumerate(w.cameras)])
    targets = img.clone() + torch.from_numpy(noise).to(dev)
    dL = torch.empty_like(img)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    tf = fr.pixel_buffer()
    nl = fr.pixel_buffer(torch.int32)
    grads = {k: torch.empty_like(v) for k, v in scene_d.items()}
    out = {"workload": "grad: 1M splats, 8 views 1280x720, loss 0.8 L1 + 0.2 SE vs render + N(0, 0.01)",
           "instances": fr.instance_count()}
    for mode in ("store", "recompute"):
        def step():
            fr.preprocess()
            fr.bin_sort()
            if mode == "store":
                fr.render(img, tf, nl)
                fr.loss_grad(img, targets, 0.2, dL, loss)
                fr.render_backward(dL, grads, tf, nl)
            else:
                fr.render(img)
                fr.loss_grad(img, targets, 0.2, dL, loss)
                fr.render_backward(dL, grads)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        D.barrier()
        a.record()
        for _ in range(args.steps):
            step()
        b.record()
        torch.cuda.synchronize()
        out[mode] = D.max_over_ranks(a.elapsed_time(b), dev) / args.steps
    out["per_pixel_bytes_stored"] = 8
    # memory of the two transmittance modes: the stored form keeps T_final (f32) and n_last (u32)
    # per pixel between the forward and the backward pass; the recomputed form keeps nothing
    out["memory_bytes"] = {"store": 8 * fr.total_pixels, "recompute": 0}
    # the backward tile kernel alone (stored transmittance), and its pair counts
    from paper_2601_14821_gb300 import _binding as B

    fr.render(img, tf, nl)
    fr.loss_grad(img, targets, 0.2, dL, loss)
    ms_k = tile_kernel_ms(B, torch, lambda: fr.render_backward(dL, grads, tf, nl), max(3, args.steps))
    pc = fr.pair_stats()
    flops = bwd_flops(pc)
    out["pairs"] = pc
    out["roofline"] = roofline_entry("render_bwd_kernel", flops, ms_k, len(w.cameras), "grad", bwd_flops(pc, strict=True))
    del fr
    out["finetune"] = finetune_run(args, dev, D, w, scene_d, cams_rec, img, targets)
    return out


def finetune_run(args, dev, D, w, scene_d, cams_rec, img, targets, iterations: int = 100) -> dict:
    """The fine-tuning loop (Section IV-F) on the gradient workload: one training view per
    iteration (seeded random order), forward, loss gradient, backward and the fused Adam step
    with the 3DGS learning rates; device-timed over ``iterations`` iterations after a warm-up."""
    import torch

    from paper_2601_14821_gb300.finetune import FineTuner

    V = len(w.cameras)
    per_view = [targets[3 * v * w.cameras[0].pixels: 3 * (v + 1) * w.cameras[0].pixels] for v in range(V)]
    params = {k: t.clone() for k, t in scene_d.items()}
    ft = FineTuner(params, cams_rec, per_view, lam=0.2, extent=4.0, device=dev, check_every=0, **CFG)
    ft.run(V, order=list(range(V)))
    first = float(ft.loss.item())
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ft.run(iterations, seed=1)
    b.record()
    torch.cuda.synchronize()
    ft.ensure_capacity()
    ms = D.max_over_ranks(a.elapsed_time(b), dev) / iterations
    return {"workload": "grad: 1M splats, 8 views 1280x720, one view per iteration", "iterations": iterations,
            "ms_per_iteration": ms, "loss_first_view0": first, "loss_last": float(ft.loss.item()),
            "lr": ft.lr}


def prune_run(args, dev, D, q: float = 0.5, iterations: int = 48) -> dict:
    """The whole iterative pruning of the scene workload: each iteration recomputes dMSE_k and
    I_k over the 16 views (preprocess, bin + sort, removal effect) and the controller removes a
    budget's worth of the splats below dMSE_MAX = 10^(-8.8 - 2q).  Targets are the render of the
    unpruned scene.  Device-timed; the controller's share is timed with events around it."""
    import torch

    import synth
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.pipeline import scene_to_device
    from paper_2601_14821_gb300.prune import PruneController

    w = synth.workload("scene")
    scene_d = scene_to_device(w.scene, dev)
    be = BatchedRemovalEffect(scene_d, synth.cameras_to_array(w.cameras), views_per_chunk=16, device=dev, **CFG)
    inst0 = be.plan()
    targets = torch.empty(3 * be.total_pixels, dtype=torch.float32, device=dev)
    be.render(targets)
    ctrl = PruneController(w.scene.n, device=dev, iterations=iterations, q=q)
    n = w.scene.n
    dmse = torch.zeros(n, dtype=torch.float64, device=dev)
    imp = torch.zeros_like(dmse)
    logits = scene_d["opacity_logits"]
    # first launches of the controller's kernels outside the timed region (on a scratch mask)
    warm = PruneController(n, device=dev, iterations=iterations, q=q)
    warm.select(dmse, imp)
    removed = torch.zeros(iterations, dtype=torch.int64, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iterations)]
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(iterations + 1)]
    torch.cuda.synchronize()
    D.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for it in range(iterations):
        starts[it].record()
        dmse.zero_()
        imp.zero_()
        be.step(targets, dmse, imp)
        ev[it][0].record()
        ctrl.select(dmse, imp)
        ctrl.apply(logits)
        ev[it][1].record()
        removed[it : it + 1].copy_(ctrl.removed)
    starts[iterations].record()
    b.record()
    torch.cuda.synchronize()
    total_ms = D.max_over_ranks(a.elapsed_time(b), dev)
    per_it = [starts[i].elapsed_time(starts[i + 1]) for i in range(iterations)]
    counts = [int(x) for x in n - np.cumsum(removed.cpu().numpy())]
    ctrl_ms = sum(x.elapsed_time(y) for x, y in ev) / iterations
    be.frames[0].preprocess()
    be.frames[0].bin_sort()
    torch.cuda.synchronize()
    sh = sh_compaction_run(args, dev, D, be.frames[0], targets, q)
    enc = codec_run(args, dev, D, scene_d, ctrl.alive, sh.pop("_sh_rgb"), w.cameras, q)
    ft = potr_ft_run(args, dev, D, enc.pop("_scene"), w.cameras, targets, q)
    return {"workload": "scene: 1M splats, 16 views 1280x720, targets = render of the unpruned scene",
            "q": q, "dmse_max": ctrl.dmse_max, "iterations": iterations,
            "ms_per_iteration": total_ms / iterations, "controller_ms_per_iteration": ctrl_ms,
            "iteration_ms": [round(x, 3) for x in per_it[:3] + per_it[-2:]],
            "splats_before": n, "splats_after": counts[-1], "alive_after_iteration": counts[:8] + counts[-2:],
            "instances_before": int(inst0), "instances_after": be.frames[0].instance_count(),
            "sh_compaction": sh, "codec": enc, "potr_ft": ft}


def codec_run(args, dev, D, scene_d, alive, sh_rgb, cams, q: float) -> dict:
    """The encoder (Section IV-E) on the pruned scene with its compacted SH coefficients: device
    part (octree, node bytes, quantised attributes) timed with CUDA events, then the stream
    assembled and zlib-coded on the host (timed on the host); the oracle's encoder on a
    20,000-splat sample for context."""
    import time

    import torch

    import synth
    from paper_2601_14821_gb300.codec import Decoder, Encoder, params
    from paper_2601_14821_gb300.compress import camera_centres

    keep = torch.nonzero(alive, as_tuple=False).flatten()
    sub = {k: t[..., keep].contiguous() for k, t in scene_d.items() if k != "sh"}
    sub["sh"] = sh_rgb[..., keep].contiguous()
    eyes = camera_centres(synth.cameras_to_array(cams))
    p = params(q)
    enc = Encoder(int(keep.numel()), dev)
    enc.run(sub, eyes, p)  # first launches outside the timed region
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record()
    for _ in range(reps):
        enc.run(sub, eyes, p)
    b.record()
    torch.cuda.synchronize()
    ms = D.max_over_ranks(a.elapsed_time(b), dev) / reps
    t0 = time.perf_counter()
    raw = enc.stream(p)
    import zlib

    packed = zlib.compress(raw, 6)
    host_ms = (time.perf_counter() - t0) * 1e3
    n = int(keep.numel())
    m, n_dups = enc.sizes()
    # the decoder on the encoder's device outputs (the decode half of a fine-tuning cycle)
    dec = Decoder(m, n, dev)
    cube = enc.cube.tolist()
    dec.run(enc.nodes, enc.dups, n_dups, enc.attrs, cube, p)
    torch.cuda.synchronize()
    dec.check()
    a.record()
    for _ in range(reps):
        dec.run(enc.nodes, enc.dups, n_dups, enc.attrs, cube, p)
    b.record()
    torch.cuda.synchronize()
    dec_ms = D.max_over_ranks(a.elapsed_time(b), dev) / reps
    t0 = time.perf_counter()
    zlib.decompress(packed)
    unzip_ms = (time.perf_counter() - t0) * 1e3
    out = {"splats": n, "device_ms": ms, "device_splats_per_s": n / (ms / 1e3), "host_stream_and_zlib_ms": host_ms,
           "decode_device_ms": dec_ms, "decode_device_splats_per_s": n / (dec_ms / 1e3), "host_unzip_ms": unzip_ms,
           "raw_bytes": len(raw), "compressed_bytes": len(packed), "bytes_per_splat": len(packed) / n,
           "node_bytes": m, "shared_leaves": n_dups, "q": q}
    if D.env_ranks()[0] == 0 and not args.no_cpu_baseline:
        from oracle import codec as ocodec

        w = synth.workload("scene")
        k = keep.cpu().numpy()[:20000]
        sample = w.scene.subset(np.isin(np.arange(w.scene.n), k))
        t0 = time.perf_counter()
        ocodec.encode(sample, eyes, p=ocodec.params(q))
        out["oracle_splats_per_s_1_core"] = sample.n / (time.perf_counter() - t0)
    out["_scene"] = sub
    return out


def potr_ft_run(args, dev, D, scene, cams, targets, q: float, cycles: int = 2, iterations: int = 500) -> dict:
    """POTR-FT (Section IV-F) on the pruned, compacted scene: R_FT = 2 cycles of encode -> decode ->
    500 fine-tuning iterations (one of the 16 views each, against the unpruned render), then the
    final encoding; every step on the device.  Reports the wall time of the cycles and final
    encoding (the raw bitstream read back), the host's zlib time apart, and the PSNR of the
    decoded scene before and after, over the 16 views."""
    import time

    import torch

    import synth
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect
    from paper_2601_14821_gb300.codec import decode, roundtrip
    from paper_2601_14821_gb300.compress import camera_centres
    from paper_2601_14821_gb300.finetune import potr_ft

    rec = synth.cameras_to_array(cams)
    eyes = camera_centres(rec)
    P = cams[0].pixels
    per_view = [targets[3 * v * P: 3 * (v + 1) * P] for v in range(len(cams))]

    def psnr(sc):
        be = BatchedRemovalEffect(sc, rec, views_per_chunk=16, device=dev, **CFG)
        be.plan()
        img = torch.empty(3 * be.total_pixels, dtype=torch.float32, device=dev)
        be.render(img)
        mse = float(torch.mean((img - targets) ** 2).item())
        return 10.0 * np.log10(1.0 / mse)

    before, _ = roundtrip(scene, eyes, q=q)
    psnr0 = psnr(before)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = potr_ft(scene, rec, per_view, eyes, q=q, cycles=cycles, iterations=iterations, extent=4.0,
                  compress=False, **CFG)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    import zlib

    t1 = time.perf_counter()
    packed = zlib.compress(out["raw"], 6)
    zlib_s = time.perf_counter() - t1
    psnr1 = psnr(decode(packed))
    return {"cycles": cycles, "iterations_per_cycle": iterations, "wall_s": wall,
            "ms_per_iteration_incl_codec": wall * 1e3 / (cycles * iterations), "host_zlib_s": zlib_s,
            "psnr_decoded_before": psnr0, "psnr_decoded_after": psnr1, "loss_per_cycle": out["losses"],
            "compressed_bytes": len(packed)}


def sh_compaction_run(args, dev, D, frame, targets, q: float) -> dict:
    """SH energy compaction (Section IV-D) of the pruned scene over the frame's 16 views: per-view
    importances from one removal pass, then the compaction of every splat (binary64), timed with
    CUDA events; the oracle's per-splat time on a 300-splat sample for context."""
    import time

    import torch

    import synth
    from paper_2601_14821_gb300.sh_compact import compact, params

    n, V = frame.n, frame.n_views
    imp_view = torch.zeros(V * n, dtype=torch.float64, device=dev)
    dmse = torch.zeros(n, dtype=torch.float64, device=dev)
    frame.removal_effect(targets, dmse, None, imp_view=imp_view)
    p = params(q)
    compact(frame, imp_view, p=p)  # first launch outside the timed region
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    a.record()
    for _ in range(reps):
        rgb, ycocg, kept = compact(frame, imp_view, p=p)
    b.record()
    torch.cuda.synchronize()
    ms = D.max_over_ranks(a.elapsed_time(b), dev) / reps
    kept_np = kept.cpu().numpy().view(np.uint32)
    seen = kept_np[0] != 0
    ac_kept = [np.array([bin(int(x)).count("1") - 1 for x in kept_np[c + 1][seen]]) for c in range(3)]
    out = {"_sh_rgb": rgb, "splats": n, "views": V, "ms": ms, "splats_per_s": n / (ms / 1e3), "lambda": p["lam"],
           "alpha": p["alpha"], "sf": p["sf"], "splats_seen": int(seen.sum()),
           "mean_ac_kept_per_channel": [float(x.mean()) if x.size else 0.0 for x in ac_kept]}
    if D.env_ranks()[0] == 0 and not args.no_cpu_baseline:
        from oracle import sh_compact as oshc

        w = synth.workload("scene")
        iv = imp_view.cpu().numpy().reshape(V, n)
        centres = np.array([oshc.camera_centre(c) for c in w.cameras])
        sample = np.nonzero(seen)[0][:300]
        t0 = time.perf_counter()
        for k in sample:
            oshc.compact_splat(w.scene.sh[:, :, k], w.scene.means[:, k], centres, iv[:, k], p["lam"], p["alpha"],
                               p["sf"])
        dt = time.perf_counter() - t0
        out["oracle_splats_per_s_1_core"] = len(sample) / dt
    return out


def multiview_config(args, dev, D, name: str, views_per_chunk, fwd_bwd: bool = False, per_view: bool = False) -> dict:
    """A many-view workload (``batched``: 3M splats, 200 views of mixed resolution; ``large``: 6M
    splats, 300 views 1920x1080): the autotuner picks the tile shape and splat batch on the first
    chunk, then whole passes over every view run chunk by chunk (``views_per_chunk`` None: every
    view in one frame, one launch per stage), eagerly and as one CUDA graph; with ``per_view`` the
    same pass one view per launch chain; the exact pair counts give Gblend/s and the removal
    kernel's roofline (kernel timed alone on the first chunk).  Steps: min(--steps, 3) per form."""
    import torch

    import synth
    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300.batched import BatchedRemovalEffect, autotune
    from paper_2601_14821_gb300.pipeline import RemovalEffectFrame, scene_to_device

    w = synth.workload(name)
    rec = synth.cameras_to_array(w.cameras)
    vpc = int(views_per_chunk or len(w.cameras))
    scene_d = scene_to_device(w.scene, dev)
    tuned = autotune(scene_d, rec, probe_views=min(vpc, 16), steps=2, warmup=1, device=dev)
    cfg = dict(tile_w=tuned["tile_w"], tile_h=tuned["tile_h"], batch=tuned["batch"])
    # targets: render of the scene with 5 % of the splats dropped + N(0, 0.01) (seeded, on device)
    keep = synth.target_drop_mask(w.scene.n, w.target_drop, w.seed)
    tb = BatchedRemovalEffect(scene_to_device(w.scene.subset(keep), dev), rec, min(vpc, 16), device=dev,
                              with_importance=False, **cfg)
    tb.plan()
    targets = torch.empty(3 * tb.total_pixels, dtype=torch.float32, device=dev)
    tb.render(targets)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed)
    targets += w.target_noise * torch.randn(targets.shape, generator=gen, device=dev)
    del tb
    torch.cuda.empty_cache()
    world = D.env_ranks()[2]
    steps = max(1, min(args.steps, 3))

    def timed(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        D.barrier()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return D.max_over_ranks(a.elapsed_time(b), dev) / reps

    out = {"workload": name, "n_splats": w.scene.n, "views_per_gpu": len(w.cameras), "views_per_chunk": vpc,
           "tuned": {k: tuned[k] for k in ("tile_w", "tile_h", "batch", "ms_per_view")},
           "autotune_table": tuned["table"], "steps": steps}
    dmse = torch.zeros(w.scene.n, dtype=torch.float64, device=dev)
    imp = torch.zeros_like(dmse)
    if per_view:
        pv = BatchedRemovalEffect(scene_d, rec, 1, device=dev, **cfg)
        pv.plan()
        pv.step(targets, dmse, imp)
        ms = timed(lambda: pv.step(targets, dmse, imp), steps)
        out["per_view_pass_ms"] = ms
        out["per_view_views_per_s"] = world * len(w.cameras) / (ms / 1e3)
        del pv
        torch.cuda.empty_cache()
    be = BatchedRemovalEffect(scene_d, rec, vpc, device=dev, **cfg)
    n_inst = be.plan()
    be.step(targets, dmse, imp)
    eager_ms = timed(lambda: be.step(targets, dmse, imp), steps)
    graph_ms = None
    try:
        g = be.capture(targets, dmse, imp)
        g.replay()
        graph_ms = timed(g.replay, steps)
        del g
    except Exception as exc:
        graph_ms = f"capture failed: {exc}"
    # exact pair counts over every chunk; the removal kernel of the first chunk timed alone
    pc = {}
    for f in be.frames:
        f.preprocess()
        f.bin_sort()
        for k2, v2 in f.pair_stats().items():
            pc[k2] = pc.get(k2, 0) + v2
    f0 = be.frames[0]
    f0.preprocess()
    f0.bin_sort()
    t0 = targets[: 3 * f0.total_pixels]
    pc0 = f0.pair_stats()
    ms_k = tile_kernel_ms(B, torch, lambda: f0.removal_effect(t0, dmse, imp, n_views_total=len(w.cameras)), steps)
    flops0 = removal_flops(pc0)
    out.update({"instances": int(n_inst), "pass_ms": eager_ms, "views_per_s": world * be.n_views / (eager_ms / 1e3),
                "graph_pass_ms": graph_ms,
                "graph_views_per_s": world * be.n_views / (graph_ms / 1e3) if isinstance(graph_ms, float) else None,
                "gblend_per_s_pass": world * (pc["examined"] + pc["back_positions"]) / (eager_ms / 1e3) / 1e9,
                "pairs": pc, "pool_gb": be.pool.nbytes() / 1e9,
                "roofline_first_chunk": roofline_entry("removal_kernel", flops0, ms_k, f0.n_views, name,
                                                       removal_flops(pc0, strict=True))})
    del be, f0
    torch.cuda.empty_cache()
    if fwd_bwd:
        # one fine-tuning step on an 8-view minibatch of the workload
        fr = RemovalEffectFrame(scene_d, rec[:8], device=dev, with_importance=False, **cfg)
        fr.plan()
        img = fr.image_buffer()
        dL = torch.empty_like(img)
        tgt = targets[: 3 * fr.total_pixels]
        tf = fr.pixel_buffer()
        nl = fr.pixel_buffer(torch.int32)
        grads = {k: torch.empty_like(v) for k, v in scene_d.items()}

        def st():
            fr.preprocess()
            fr.bin_sort()
            fr.render(img, tf, nl)
            fr.loss_grad(img, tgt, 0.2, dL)
            fr.render_backward(dL, grads, tf, nl)

        st()
        out["fwd_bwd_ms_per_step_8_views"] = timed(st, steps)
        del fr
        torch.cuda.empty_cache()
    return out


def scene_config(n_splats: int, n_views: int, world: int) -> dict:
    """The timed workload, named the same way on both arms."""
    return {"workload": "scene: 1M splats (70% unit ball, 30% shell 2-10), 16 views 1280x720 on a ring "
                        "of radius 4, targets = render with 5% of splats dropped + N(0, 0.01)",
            "n_splats": int(n_splats), "views_per_gpu": int(n_views), "resolution": "1280x720",
            "tile": f"{CFG['tile_w']}x{CFG['tile_h']}", "splat_batch": CFG["batch"],
            "l2": "inputs larger than L2 (236 MB parameters, 0.77 GB raster records, 0.45 GB instances)",
            "parallelism": f"views replicated per GPU x{world}"}


# ------------------------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ------------------------------------------------------------------------------------------

def run_reference(args):
    """The CPU oracle as it stands, on the same workload: each step is one frame of all the
    workload's views on every host core (views concurrently, see oracle_frame_seconds)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth

    w = synth.workload(WORKLOAD)
    n_views = len(w.cameras)
    cores = host_cores()
    views = list(range(n_views))
    targets = oracle_targets(w, views, cores)
    for _ in range(args.warmup):
        oracle_frame_seconds(w, views, targets, cores)
    tot = 0.0
    for _ in range(args.steps):
        tot += oracle_frame_seconds(w, views, targets, cores)
    value = n_views * args.steps / tot
    line = {"metric": METRIC, "value": value, "unit": "views/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": scene_config(w.scene.n, n_views, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step all {n_views} views of the workload on {cores} host threads "
                                       "(views concurrently; dMSE_k / I_k added in view order)"},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
