"""POTR codec (Section IV-E) driven from the device.

``potr_codec_encode`` builds the octree, its depth-first node bytes, the table of shared
depth-limit leaves and the quantised attributes; ``potr_codec_decode`` inverts them into a scene.
This module lays them out as the bitstream (header, node bytes, table, attributes property after
property, little-endian) and entropy codes it on the host with zlib (the paper uses zstd, which
this image does not have).  ``roundtrip`` takes a scene through the encoder and the decoder
without leaving the device (the bitstream is lossless after quantisation), the decode and encode
halves of a POTR-FT cycle (Section IV-F).
"""
from __future__ import annotations

import struct
import zlib

import numpy as np
import torch

from . import _binding as B
from .pipeline import scene_struct

MAGIC = b"POTR"
VERSION = 1
HEADER = 80  # magic, version, n, corner, edge, four scale factors, node count


def params(q: float) -> dict:
    return {"sf_scale": 1.0 + 4000.0 * q, "sf_rotation": 1.0 + 400.0 * q, "sf_opacity": 1.0 + 200.0 * q,
            "sf_sh": 1.0 + 100.0 * q, "beta": 1.4e-4 * q, "gamma": 5.0 * 10.0 ** (-3.0 - 5.0 * q)}


def _cparams(p: dict):
    return B.CodecParams(p["sf_scale"], p["sf_rotation"], p["sf_opacity"], p["sf_sh"], p.get("beta", 0.0),
                         p.get("gamma", 0.0))


def _check_status(status: torch.Tensor, what: str):
    code = int(status[0].item())
    if code != B.POTR_OK:
        raise B.PotrError(what, code)


class Encoder:
    """Device buffers of the encoder for scenes of n splats."""

    def __init__(self, n: int, device="cuda"):
        self.n = int(n)
        self.device = torch.device(device)
        self.ws = torch.empty(B.potr_codec_workspace_size(self.n), dtype=torch.uint8, device=self.device)
        self.nodes = torch.empty(22 * self.n, dtype=torch.uint8, device=self.device)
        self.dups = torch.empty(max(self.n, 2), dtype=torch.int32, device=self.device)
        self.counts = torch.zeros(2, dtype=torch.int32, device=self.device)  # node bytes, table pairs
        self.order = torch.empty(self.n, dtype=torch.int32, device=self.device)
        self.attrs = torch.empty(55 * self.n, dtype=torch.int32, device=self.device)
        self.cube = torch.empty(4, dtype=torch.float64, device=self.device)
        self.status = torch.zeros(2, dtype=torch.int64, device=self.device)

    def run(self, scene: dict, eyes, p: dict, stream=None):
        """Enqueue the device part (no host synchronisation)."""
        e = torch.as_tensor(np.ascontiguousarray(eyes, np.float64).reshape(-1, 3), device=self.device)
        self._eyes = e
        B.potr_codec_encode(scene_struct(scene), e, e.shape[0], _cparams(p), self.nodes, self.counts[0:1],
                            self.dups, self.counts[1:2], self.order, self.attrs, self.cube, self.status, self.ws,
                            stream)

    def sizes(self) -> tuple[int, int]:
        """(node bytes, table pairs) of the last run (synchronises the device)."""
        torch.cuda.synchronize(self.device)
        m, d = self.counts.tolist()
        return int(m), int(d)

    def stream(self, p: dict) -> bytes:
        """The raw bitstream of the last run (synchronises)."""
        m, d = self.sizes()
        nodes = self.nodes[:m].cpu().numpy().tobytes()
        table = self.dups[:2 * d].cpu().numpy().astype("<u4").tobytes()
        cube = self.cube.cpu().numpy()
        head = MAGIC + struct.pack("<II", VERSION, self.n) + struct.pack("<4d", *cube)
        head += struct.pack("<4d", p["sf_scale"], p["sf_rotation"], p["sf_opacity"], p["sf_sh"])
        body = self.attrs.cpu().numpy().astype("<i4").tobytes()
        return head + struct.pack("<I", m) + nodes + struct.pack("<I", d) + table + body


def encode(scene: dict, eyes, q: float = 0.5, p: dict | None = None, level: int = 6) -> dict:
    """Encode a scene: returns the raw and the zlib-compressed bitstream and the leaf order."""
    p = p or params(q)
    enc = Encoder(int(scene["means"].shape[-1]), scene["means"].device)
    enc.run(scene, eyes, p)
    raw = enc.stream(p)
    return {"raw": raw, "compressed": zlib.compress(raw, level), "order": enc.order.cpu().numpy()}


def empty_scene(n: int, device) -> dict:
    """Scene-shaped float32 planes (means [3][n], log_scales [3][n], quats [4][n],
    opacity_logits [n], sh [16][3][n])."""
    f = dict(dtype=torch.float32, device=device)
    return {"means": torch.empty(3, n, **f), "log_scales": torch.empty(3, n, **f), "quats": torch.empty(4, n, **f),
            "opacity_logits": torch.empty(n, **f), "sh": torch.empty(16, 3, n, **f)}


class Decoder:
    """Device buffers of the decoder; ``run`` enqueues potr_codec_decode into ``self.scene``."""

    def __init__(self, n_nodes: int, n: int, device="cuda"):
        self.n_nodes, self.n = int(n_nodes), int(n)
        self.device = torch.device(device)
        self.ws = torch.empty(B.potr_codec_decode_workspace_size(self.n_nodes, self.n), dtype=torch.uint8,
                              device=self.device)
        self.status = torch.zeros(2, dtype=torch.int64, device=self.device)
        self.scene = empty_scene(self.n, self.device)

    def run(self, nodes, dups, n_dups: int, attrs, cube, p: dict, stream=None):
        B.potr_codec_decode(nodes, self.n_nodes, dups, n_dups, attrs, self.n, cube, _cparams(p), self.scene,
                            self.status, self.ws, stream)

    def check(self):
        _check_status(self.status, "potr_codec_decode")


def parse(raw: bytes) -> dict:
    """Header fields and the byte ranges of a raw (decompressed) bitstream."""
    if raw[:4] != MAGIC:
        raise ValueError("not a POTR bitstream")
    version, n = struct.unpack_from("<II", raw, 4)
    cube = struct.unpack_from("<4d", raw, 12)
    sf = struct.unpack_from("<4d", raw, 44)
    (m,) = struct.unpack_from("<I", raw, 76)
    (d,) = struct.unpack_from("<I", raw, HEADER + m)
    body = HEADER + m + 4 + 8 * d
    if len(raw) != body + 4 * 55 * n:
        raise ValueError("truncated POTR bitstream")
    return {"version": version, "n": n, "cube": cube, "n_nodes": m, "n_dups": d,
            "p": {"sf_scale": sf[0], "sf_rotation": sf[1], "sf_opacity": sf[2], "sf_sh": sf[3]},
            "nodes": (HEADER, HEADER + m), "dups": (HEADER + m + 4, body), "attrs": (body, len(raw))}


def decode(stream: bytes, device="cuda", compressed: bool = True) -> dict:
    """Decode a bitstream into a scene of device tensors (splats in stream order)."""
    raw = zlib.decompress(stream) if compressed else stream
    h = parse(raw)
    dev = torch.device(device)

    def up(rng, dtype):
        a = np.frombuffer(raw[rng[0]:rng[1]], dtype).copy()
        return torch.as_tensor(a, device=dev)

    nodes = up(h["nodes"], np.uint8)
    dups = up(h["dups"], "<i4") if h["n_dups"] else None
    attrs = up(h["attrs"], "<i4")
    dec = Decoder(h["n_nodes"], h["n"], dev)
    dec.run(nodes, dups, h["n_dups"], attrs, h["cube"], h["p"])
    dec.check()
    return dec.scene


def roundtrip(scene: dict, eyes, q: float = 0.5, p: dict | None = None, stream=None) -> tuple[dict, torch.Tensor]:
    """Encode and decode on the device: returns the decoded scene (splats in leaf order) and the
    leaf order.  One host synchronisation, to size the decoder."""
    p = p or params(q)
    dev = scene["means"].device
    enc = Encoder(int(scene["means"].shape[-1]), dev)
    enc.run(scene, eyes, p, stream)
    m, d = enc.sizes()
    _check_status(enc.status, "potr_codec_encode")
    cube = enc.cube.tolist()
    dec = Decoder(m, enc.n, dev)
    dec.run(enc.nodes, enc.dups, d, enc.attrs, cube, p, stream)
    dec.check()
    return dec.scene, enc.order
