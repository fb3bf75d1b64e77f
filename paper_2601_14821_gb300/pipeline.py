"""Frame-level driver of the C ABI: buffer ownership (torch device memory), instance-capacity
planning, and the preprocess -> bin_sort -> render / removal_effect chain on one stream.

A *frame* is a set of views processed together (one view for the per-view form, many for
the batched form).  ``RemovalEffectFrame`` holds every buffer the chain needs, so a step is a
fixed sequence of asynchronous C calls that can be replayed or captured in a CUDA graph.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _binding as B

SCENE_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def scene_to_device(scene, device="cuda") -> dict:
    """synth.Scene (numpy SoA planes) -> dict of contiguous float32 device tensors."""
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).to(device) for k in SCENE_KEYS}


def scene_struct(sc: dict) -> B.Scene:
    return B.Scene(sc["means"].data_ptr(), sc["log_scales"].data_ptr(), sc["quats"].data_ptr(),
                   sc["opacity_logits"].data_ptr(), sc["sh"].data_ptr(), int(sc["means"].shape[-1]))


class BufferPool:
    """Named device buffers shared by frames that run one after another on one stream (the view
    chunks of a batched pass).  ``get`` returns a typed view of the named buffer, growing it when
    a caller needs more; frames re-take their views (``rebind``) once every frame is planned, so
    nothing is reallocated while steps run or a CUDA graph replays."""

    def __init__(self, device):
        self.device = torch.device(device)
        self.store: dict[str, torch.Tensor] = {}

    def get(self, name: str, numel: int, dtype) -> torch.Tensor:
        esize = torch.empty(0, dtype=dtype).element_size()
        nbytes = max(int(numel), 1) * esize
        t = self.store.get(name)
        if t is None or t.numel() < nbytes:
            t = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.store[name] = t
        return t[:nbytes].view(dtype)

    def nbytes(self) -> int:
        return sum(t.numel() for t in self.store.values())


class RemovalEffectFrame:
    """All device buffers for one frame (scene x views) and the C calls over them."""

    def __init__(self, scene: dict, cams_rec: np.ndarray, device="cuda", capacity: int | None = None,
                 with_importance: bool = True, schedule: bool = True, pool: BufferPool | None = None, **cfg):
        self.device = torch.device(device)
        self.scene = scene
        self.scene_c = scene_struct(scene)
        self.n = int(scene["means"].shape[-1])
        self.cams_rec = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)
        self.n_views = self.cams_rec.shape[0]
        self.cfg = B.make_config(**cfg)
        info, self.total_tiles, self.total_pixels = B.potr_view_layout(self.cams_rec, self.cfg)
        self.info_np = info.view(np.dtype([("width", "<i4"), ("height", "<i4"), ("tiles_x", "<i4"),
                                           ("tiles_y", "<i4"), ("tile_base", "<i8"), ("pixel_base", "<i8")]))
        dev = self.device
        self.d_cams = torch.from_numpy(self.cams_rec.copy()).to(dev)
        self.d_info = torch.from_numpy(info.copy()).to(dev)
        self.frame = B.Frame(self.d_cams.data_ptr(), self.d_info.data_ptr(), self.n_views, self.total_tiles,
                             self.total_pixels)
        self.pool = pool if pool is not None else BufferPool(dev)
        self.cov3d = torch.empty(6 * self.n, dtype=torch.float32, device=dev)
        self.opacity = torch.empty(self.n, dtype=torch.float32, device=dev)
        self.n_instances = torch.zeros(1, dtype=torch.int32, device=dev)
        self.status = torch.zeros(2, dtype=torch.int64, device=dev)
        self.pre_status = torch.zeros(2, dtype=torch.int64, device=dev)  # non-finite splats (potr_preprocess)
        self.sched_ws = torch.empty(B.potr_tile_schedule_workspace_size(), dtype=torch.uint8, device=dev)
        self.schedule = schedule
        self.with_importance = with_importance
        self.capacity = int(capacity) if capacity else 1
        self.rebind()

    # -------------------------------------------------------------------------------------
    def rebind(self):
        """(Re)take every pooled buffer at the current sizes and rebuild the C views."""
        vn = self.n_views * self.n
        i32, P = torch.int32, self.pool
        self.raster = P.get("raster", vn * 12, torch.float32)
        self.cull = P.get("cull", vn * 4, i32)
        self.depth = P.get("depth", vn, torch.float32)
        self.rect = P.get("rect", 2 * vn, i32)
        self.touched = P.get("touched", vn, i32)
        self.offsets = P.get("offsets", vn, i32)
        self.ranges = P.get("ranges", 2 * self.total_tiles, i32)
        # longest-list-first tile order for the persistent tile kernels (+1 work-counter word)
        self.order = P.get("order", self.total_tiles + 1, i32) if self.schedule else None
        self.views = B.Views(self.cov3d.data_ptr(), self.opacity.data_ptr(), self.raster.data_ptr(),
                             self.depth.data_ptr(), self.rect.data_ptr(), self.touched.data_ptr(),
                             self.offsets.data_ptr(), self.n_instances.data_ptr(), self.cull.data_ptr())
        self._alloc(self.capacity)

    def _alloc(self, capacity: int):
        P = self.pool
        self.capacity = int(capacity)
        self.tiles = P.get("tiles", self.capacity, torch.int32)  # sorted instances' global tiles
        self.vals = P.get("vals", self.capacity, torch.int32)
        self.ws = P.get("sort_ws", B.potr_bin_sort_workspace_size(self.n, self.n_views, self.total_tiles,
                                                                   self.capacity), torch.uint8)
        self.inst_dse = P.get("inst_dse", self.capacity, torch.float32)
        self.inst_imp = P.get("inst_imp", self.capacity, torch.float32) if self.with_importance else None

    def plan(self, slack: float = 1.05) -> int:
        """Run preprocess + binning once, grow the instance capacity to fit, return the count."""
        self.preprocess()
        self.bin_sort()
        torch.cuda.synchronize(self.device)
        code, need = self.status.tolist()
        if code == B.POTR_ERR_CAPACITY:
            self._alloc(max(int(need * slack) + 1024, 1024))
            self.bin_sort()
            torch.cuda.synchronize(self.device)
            code, need = self.status.tolist()
        if code != 0:
            raise B.PotrError("potr_bin_sort (device)", int(code))
        return self.instance_count()

    def instance_count(self) -> int:
        return int(self.n_instances.cpu().numpy().view(np.uint32)[0])

    # -------------------------------------------------------------------------------------
    def preprocess(self, stream=None):
        self.pre_status.zero_()
        B.potr_preprocess(self.scene_c, self.frame, self.cfg, self.views, stream, status=self.pre_status)

    def nonfinite(self) -> tuple[int, int]:
        """(status code, splats culled for non-finite parameters) of the last preprocess (synchronises)."""
        w = self.pre_status.cpu().numpy().view(np.int32)
        return int(w[0]), int(w[1])

    def bin_sort(self, stream=None):
        """Binning + sort, then (with scheduling on) the longest-list-first tile order."""
        self._sort_gen = getattr(self, "_sort_gen", 0) + 1
        self.status.zero_()
        B.potr_bin_sort(self.views, self.frame, self.cfg, self.n, self.capacity, self.tiles, self.vals, self.ranges,
                        self.status, self.ws, stream)
        if self.schedule:
            B.potr_tile_schedule(self.frame, self.ranges, self.order, self.sched_ws, stream)

    def render(self, images=None, t_final=None, n_last=None, stream=None):
        B.potr_render(self.views, self.frame, self.cfg, self.n, self.vals, self.ranges, images, t_final, n_last, stream,
                      order=self.order)

    def removal_effect(self, targets, dmse, importance=None, n_views_total=None, dsse_view=None, images=None,
                       stream=None, imp_view=None):
        want_imp = importance is not None or imp_view is not None
        ws = self.pool.get("removal_ws", B.potr_removal_workspace_size(self.capacity, self.total_tiles, want_imp),
                           torch.uint8)
        B.potr_removal_effect(self.views, self.frame, self.cfg, self.n, self.vals, self.ranges, targets,
                              int(n_views_total or self.n_views), self.capacity, self.inst_dse,
                              self.inst_imp if want_imp else None, dmse, importance, dsse_view,
                              images, stream, order=self.order, imp_view=imp_view, ws=ws)

    def bind_scene(self, scene: dict):
        """Point the frame at other parameter tensors of the same size (e.g. autograd inputs)."""
        assert int(scene["means"].shape[-1]) == self.n
        self.scene = scene
        self.scene_c = scene_struct(scene)

    def status_code(self) -> int:
        """Device status of the last binning (synchronises)."""
        return int(self.status[0].item())

    def loss_grad(self, images, targets, lam: float, dL_dimages, loss=None, stream=None):
        ws = None
        if loss is not None:
            ws = getattr(self, "_loss_ws", None)
            if ws is None:
                ws = self._loss_ws = torch.empty(B.potr_loss_workspace_size(self.total_pixels), dtype=torch.uint8,
                                                 device=self.device)
        B.potr_loss_grad(self.frame, images, targets, lam, loss, dL_dimages, ws, stream)

    def render_backward(self, dL_dimages, grads: dict, t_final=None, n_last=None, stream=None):
        """Parameter gradients (dict of tensors shaped like the scene, overwritten)."""
        ws = self.pool.get("bwd_ws", B.potr_render_backward_workspace_size(self.capacity, self.n_views * self.n),
                           torch.uint8)
        g = B.SceneGrads(*(grads[k].data_ptr() for k in SCENE_KEYS))
        B.potr_render_backward(self.scene_c, self.views, self.frame, self.cfg, self.vals, self.ranges, t_final, n_last,
                               dL_dimages, self.capacity, g, ws, stream, order=self.order)

    def pair_stats(self, stream=None) -> dict:
        """Exact pair counts of the forward and removal walks (see potr_pair_stats)."""
        counts = torch.zeros(5, dtype=torch.int64, device=self.device)
        B.potr_pair_stats(self.views, self.frame, self.cfg, self.n, self.vals, self.ranges, counts, stream)
        c = [int(x) for x in counts.cpu().tolist()]
        return dict(examined=c[0], passed=c[1], composited=c[2], back_positions=c[3], back_passed=c[4])

    def step(self, targets, dmse, importance=None, n_views_total=None, stream=None):
        """One pass of the whole path: preprocess, bin + sort, removal effect + per-splat reduce."""
        self.preprocess(stream)
        self.bin_sort(stream)
        self.removal_effect(targets, dmse, importance, n_views_total, stream=stream)

    def image_buffer(self):
        return torch.empty(3 * self.total_pixels, dtype=torch.float32, device=self.device)

    def pixel_buffer(self, dtype=torch.float32):
        return torch.empty(self.total_pixels, dtype=dtype, device=self.device)

    def view_image(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        """[3, H, W] view of view v inside a packed per-frame image buffer."""
        vi = self.info_np[v]
        h, w, pb = int(vi["height"]), int(vi["width"]), int(vi["pixel_base"])
        return flat[3 * pb: 3 * pb + 3 * h * w].view(3, h, w)

    def view_pixels(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        vi = self.info_np[v]
        h, w, pb = int(vi["height"]), int(vi["width"]), int(vi["pixel_base"])
        return flat[pb: pb + h * w].view(h, w)


class HostPipeline:
    """Removal-effect steps whose inputs arrive in pinned host memory and whose results go back
    to it, with the transfers overlapped with compute: the parameters and targets of step i + 1
    are copied to the device (on a copy stream) while step i computes, and step i's dMSE_k /
    I_k are copied back while step i + 1 computes.  Device inputs and outputs are double
    buffered; events order every copy against the compute that uses or produces its buffer."""

    def __init__(self, frame: RemovalEffectFrame):
        self.frame = frame
        dev = frame.device
        self.compute = torch.cuda.current_stream(dev)
        self.copy = torch.cuda.Stream(device=dev)
        self.scenes = [{k: torch.empty_like(t) for k, t in frame.scene.items()} for _ in range(2)]
        self.targets = [torch.empty(3 * frame.total_pixels, dtype=torch.float32, device=dev) for _ in range(2)]
        self.dmse = [torch.zeros(frame.n, dtype=torch.float64, device=dev) for _ in range(2)]
        self.imp = [torch.zeros(frame.n, dtype=torch.float64, device=dev) for _ in range(2)]
        self.inputs_ready = [torch.cuda.Event() for _ in range(2)]
        self.done = [torch.cuda.Event() for _ in range(2)]
        self.read = [torch.cuda.Event() for _ in range(2)]
        self.i = 0   # steps run
        self.up = 0  # input sets uploaded

    def upload(self, host_scene: dict, host_targets: torch.Tensor):
        """Queue the copy of the inputs of the next step not yet uploaded (pinned host tensors)."""
        s = self.up % 2
        self.up += 1
        with torch.cuda.stream(self.copy):
            self.copy.wait_event(self.done[s])  # the step that last read this set has finished
            for k, t in host_scene.items():
                self.scenes[s][k].copy_(t, non_blocking=True)
            self.targets[s].copy_(host_targets, non_blocking=True)
            self.inputs_ready[s].record(self.copy)

    def step(self, host_dmse: torch.Tensor, host_imp: torch.Tensor):
        """Run the step on the uploaded inputs and queue the copy of its results to the host."""
        if self.i >= self.up:
            raise RuntimeError("upload the step's inputs first")
        s = self.i % 2
        f = self.frame
        self.compute.wait_event(self.inputs_ready[s])
        self.compute.wait_event(self.read[s])  # the results of two steps ago have left this set
        f.bind_scene(self.scenes[s])
        self.dmse[s].zero_()
        self.imp[s].zero_()
        f.step(self.targets[s], self.dmse[s], self.imp[s])
        self.done[s].record(self.compute)
        with torch.cuda.stream(self.copy):
            self.copy.wait_event(self.done[s])
            host_dmse.copy_(self.dmse[s], non_blocking=True)
            host_imp.copy_(self.imp[s], non_blocking=True)
            self.read[s].record(self.copy)
        self.i += 1

    def join(self):
        """Make the compute stream wait for every queued copy (no host synchronisation)."""
        self.compute.wait_stream(self.copy)

    def finish(self):
        self.join()
        self.compute.synchronize()
