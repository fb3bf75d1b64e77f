"""POTR encoder (Section IV-E) driven from the device: ``potr_codec_encode`` builds the octree,
its depth-first node bytes and the quantised attributes; this module lays them out as the
bitstream (header, node bytes, attributes property after property, little-endian) and entropy
codes it on the host with zlib (the paper uses zstd, which this image does not have)."""
from __future__ import annotations

import struct
import zlib

import numpy as np
import torch

from . import _binding as B
from .pipeline import scene_struct

MAGIC = b"POTR"
VERSION = 1


def params(q: float) -> dict:
    return {"sf_scale": 1.0 + 4000.0 * q, "sf_rotation": 1.0 + 400.0 * q, "sf_opacity": 1.0 + 200.0 * q,
            "sf_sh": 1.0 + 100.0 * q, "beta": 1.4e-4 * q, "gamma": 5.0 * 10.0 ** (-3.0 - 5.0 * q)}


class Encoder:
    """Device buffers of the encoder for scenes of n splats."""

    def __init__(self, n: int, device="cuda"):
        self.n = int(n)
        self.device = torch.device(device)
        self.ws = torch.empty(B.potr_codec_workspace_size(self.n), dtype=torch.uint8, device=self.device)
        self.nodes = torch.empty(22 * self.n, dtype=torch.uint8, device=self.device)
        self.n_nodes = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.order = torch.empty(self.n, dtype=torch.int32, device=self.device)
        self.attrs = torch.empty(55 * self.n, dtype=torch.int32, device=self.device)
        self.cube = torch.empty(4, dtype=torch.float64, device=self.device)
        self.status = torch.zeros(2, dtype=torch.int64, device=self.device)

    def run(self, scene: dict, eyes, p: dict, stream=None):
        """Enqueue the device part (no host synchronisation)."""
        e = torch.as_tensor(np.ascontiguousarray(eyes, np.float64).reshape(-1, 3), device=self.device)
        self._eyes = e
        cp = B.CodecParams(p["sf_scale"], p["sf_rotation"], p["sf_opacity"], p["sf_sh"], p["beta"], p["gamma"])
        B.potr_codec_encode(scene_struct(scene), e, e.shape[0], cp, self.nodes, self.n_nodes, self.order, self.attrs,
                            self.cube, self.status, self.ws, stream)

    def stream(self, p: dict) -> bytes:
        """The raw bitstream of the last run (synchronises)."""
        m = int(self.n_nodes.item())
        nodes = self.nodes[:m].cpu().numpy().tobytes()
        cube = self.cube.cpu().numpy()
        head = MAGIC + struct.pack("<II", VERSION, self.n) + struct.pack("<4d", *cube)
        head += struct.pack("<4d", p["sf_scale"], p["sf_rotation"], p["sf_opacity"], p["sf_sh"])
        body = self.attrs.cpu().numpy().astype("<i4").tobytes()
        return head + struct.pack("<I", m) + nodes + body


def encode(scene: dict, eyes, q: float = 0.5, p: dict | None = None, level: int = 6) -> dict:
    """Encode a scene: returns the raw and the zlib-compressed bitstream and the leaf order."""
    p = p or params(q)
    enc = Encoder(int(scene["means"].shape[-1]), scene["means"].device)
    enc.run(scene, eyes, p)
    raw = enc.stream(p)
    return {"raw": raw, "compressed": zlib.compress(raw, level), "order": enc.order.cpu().numpy()}
