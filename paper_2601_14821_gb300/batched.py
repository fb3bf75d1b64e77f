"""Batched removal effect over many views, and the tile-shape autotuner.

The removal effect is summed over every view (Section IV-B), so a pass over hundreds of views of
uneven resolution is split into view chunks; each chunk is one frame (one launch per stage
over all of its views, tiles of every view in one persistent grid) and every chunk shares one
pool of device buffers, run back to back on one stream.  The per-splat dMSE_k / I_k add view by
view in view order, so the result does not depend on the chunking.  A whole pass can be
captured as one CUDA graph and replayed.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from .pipeline import BufferPool, RemovalEffectFrame


class BatchedRemovalEffect:
    def __init__(self, scene: dict, cams_rec: np.ndarray, views_per_chunk: int = 16, device="cuda",
                 with_importance: bool = True, **cfg):
        cams_rec = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)
        self.device = torch.device(device)
        self.n_views = cams_rec.shape[0]
        self.views_per_chunk = int(views_per_chunk)
        self.pool = BufferPool(self.device)
        self.frames = [RemovalEffectFrame(scene, cams_rec[i:i + views_per_chunk], device=self.device, pool=self.pool,
                                          with_importance=with_importance, **cfg)
                       for i in range(0, self.n_views, views_per_chunk)]
        self.total_pixels = sum(f.total_pixels for f in self.frames)
        self.graph = None

    @property
    def n(self) -> int:
        return self.frames[0].n

    def plan(self, slack: float = 1.05) -> int:
        """Size the shared instance buffers for the largest chunk; returns the total instance count."""
        total = 0
        for f in self.frames:
            total += f.plan(slack)
        cap = max(f.capacity for f in self.frames)
        for f in self.frames:
            f.capacity = cap
            f.rebind()
        return total

    def set_batch(self, batch: int):
        for f in self.frames:
            f.cfg.batch = int(batch)

    def step(self, targets: torch.Tensor, dmse: torch.Tensor, importance: torch.Tensor | None = None, stream=None):
        """One pass over every view: per chunk preprocess, bin + sort, removal effect."""
        off = 0
        for f in self.frames:
            t = targets[3 * off: 3 * (off + f.total_pixels)]
            f.step(t, dmse, importance, n_views_total=self.n_views, stream=stream)
            off += f.total_pixels

    def render(self, images: torch.Tensor, stream=None):
        """Render every view into a packed image buffer (3 * total_pixels floats)."""
        off = 0
        for f in self.frames:
            f.preprocess(stream)
            f.bin_sort(stream)
            f.render(images[3 * off: 3 * (off + f.total_pixels)], stream=stream)
            off += f.total_pixels

    def capture(self, targets, dmse, importance=None) -> torch.cuda.CUDAGraph:
        """CUDA graph of one whole pass (warmed up on a side stream first)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.step(targets, dmse, importance)
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(targets, dmse, importance)
        self.graph = g
        return g


TILE_SHAPES = ((16, 16), (8, 32), (32, 8))
SPLAT_BATCHES = (256,)  # the kernels no longer depend on the config field
_CACHE: dict = {}


def _signature(scene: dict, cams_rec: np.ndarray) -> str:
    sizes = sorted({(int(w), int(h)) for w, h in cams_rec.reshape(-1, 18)[:, 16:18].view(np.int32)})
    n = int(scene["means"].shape[-1])
    return f"{torch.cuda.get_device_name()}|n~{1 << max(0, n.bit_length() - 1)}|{sizes}"


def autotune(scene: dict, cams_rec: np.ndarray, probe_views: int = 16, steps: int = 3, warmup: int = 2,
             device="cuda", cache_path: str | None = None, tiles=TILE_SHAPES, batches=SPLAT_BATCHES) -> dict:
    """Time one removal-effect pass (preprocess, bin + sort, removal) over the first
    ``probe_views`` views for every tile shape x splat batch, and return the fastest as
    {"tile_w", "tile_h", "batch", "ms_per_view", "table"}.  Results are cached per GPU model,
    splat-count bucket and view resolutions (in memory, and in ``cache_path`` when given)."""
    cams = np.ascontiguousarray(cams_rec, np.float32).reshape(-1, 18)[:probe_views]
    key = _signature(scene, cams)
    if key not in _CACHE and cache_path and os.path.exists(cache_path):
        _CACHE.update(json.load(open(cache_path)))
    if key in _CACHE:
        return _CACHE[key]
    dev = torch.device(device)
    table = []
    dmse = torch.zeros(int(scene["means"].shape[-1]), dtype=torch.float64, device=dev)
    imp = torch.zeros_like(dmse)
    for tw, th in tiles:
        fr = RemovalEffectFrame(scene, cams, device=dev, tile_w=tw, tile_h=th, batch=256)
        fr.plan()
        tg = torch.full((3 * fr.total_pixels,), 0.3, dtype=torch.float32, device=dev)
        for b in batches:
            fr.cfg.batch = int(b)
            for _ in range(warmup):
                fr.step(tg, dmse, imp)
            torch.cuda.synchronize(dev)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(steps):
                fr.step(tg, dmse, imp)
            z.record()
            torch.cuda.synchronize(dev)
            table.append({"tile_w": tw, "tile_h": th, "batch": b,
                          "ms_per_view": a.elapsed_time(z) / steps / cams.shape[0]})
        del fr
    best = min(table, key=lambda r: r["ms_per_view"])
    out = dict(best, table=table, when=time.time())
    _CACHE[key] = out
    if cache_path:
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(_CACHE, open(cache_path, "w"))
    return out
