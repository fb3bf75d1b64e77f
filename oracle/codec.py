"""POTR codec, encoder side (Section IV-E "Codec") -- plain reference.

TEST INFRASTRUCTURE ONLY: loaded by the tests and the benchmark's CPU baseline; the CUDA
library never calls it and shares no code with it.

What the section fixes:
  * attributes (scale, rotation, opacity, SH coefficients) are quantised uniformly,
    x^ = floor(1/2 + x SF), and dequantised x~ = x^ / SF, with one scale factor per attribute
    (SF_SH = 1 + 100q, SF_opacity = 1 + 200q, SF_rotation = 1 + 400q, SF_scale = 1 + 4000q);
    opacity is reconstructed off-centre, x~ = (x^ + 0.25) / SF;
  * geometry: each position is quantised to the centre of an octree leaf.  Leaves are split
    while they hold several splats or their splat fails the precision criterion
    ||mu - mu^|| < max(gamma, beta min_s ||mu - mu_s||) (mu_s the camera eyes; beta =
    1.4e-4 q, gamma = 5 10^(-3-5q));
  * the octree is serialised depth first, a node's occupancy byte (bit c set when child c
    exists) appended when the node is first visited (so a leaf appends 0); attributes follow
    in the order of that traversal (splat after splat would also do -- the section serialises property after
    property: all splats' first attribute, then the next); DC coefficients are differentially
    encoded, the real quaternion component is omitted; the stream is then entropy coded.

Readings (the section is silent on them):
  * root cube: corner = per-axis minimum of the positions, edge S = the largest per-axis
    range (1 if all coincide); a cell at depth d has edge S / 2^d; child c of a cell holds the
    octant with x offset bit (c >> 2) & 1, y bit (c >> 1) & 1, z bit c & 1 (Morton order);
    positions map to integer cells at the depth limit 21, X = floor((mu - corner) / S 2^21)
    clamped to [0, 2^21 - 1] (binary64), and a splat's cell at depth d is X >> (21 - d);
  * splitting stops at depth 21 even if several splats share the leaf (they are written in
    index order); that leaf writes 0 like every leaf, and a table after the node bytes lists
    each such leaf as (its ordinal among the leaves, splat count - 1), so every node byte is a
    plain child mask and the stream can be parsed in parallel;
  * the precision test uses binary64 with the operations in the written order; the leaf centre
    is corner + (cell + 1/2) S / 2^d per axis;
  * scale = the stored log-scales; opacity = sigmoid(logit) in [0, 1]; rotation = the
    normalised quaternion with w >= 0 (sign flipped otherwise), x, y, z stored; SH: 48
    coefficients, DC (planes 0-2) as differences of consecutive splats' quantised values in
    stream order (the first against 0);
  * decoding to a scene: the opacity logit is log(o / (1 - o)) of the dequantised opacity
    clamped to [1e-6, 1 - 1e-6] (the off-centre reconstruction can exceed 1), and the
    quaternion's real part is sqrt(max(0, 1 - x^2 - y^2 - z^2));
  * stream: little-endian; header (magic 'POTR', version, n, corner (3 x f64), S (f64), the
    four SF (f64)); the number of node bytes (u32) and the node bytes; the number of shared
    leaves (u32) and their (ordinal, count - 1) pairs (u32); then property after property over the splats in
    stream order, each quantised value as int32: 3 log-scales, 3 rotation components, opacity,
    48 SH values (coefficient-major, channel inside); entropy coding: zlib level 9 (the paper
    uses zstd, which this image does not have).
"""
from __future__ import annotations

import math
import struct
import zlib

import numpy as np

DEPTH = 21
MAGIC = b"POTR"
VERSION = 1


def params(q: float) -> dict:
    return {"sf_sh": 1.0 + 100.0 * q, "sf_opacity": 1.0 + 200.0 * q, "sf_rotation": 1.0 + 400.0 * q,
            "sf_scale": 1.0 + 4000.0 * q, "beta": 1.4e-4 * q, "gamma": 5.0 * 10.0 ** (-3.0 - 5.0 * q)}


def quantise(x, sf: float) -> np.ndarray:
    return np.floor(0.5 + np.asarray(x, np.float64) * sf).astype(np.int64)


def root_cube(means):
    mu = np.asarray(means, np.float64)
    lo = mu.min(axis=1)
    S = float((mu.max(axis=1) - lo).max())
    return lo, (S if S > 0.0 else 1.0)


def cells(means, corner, S):
    """Integer cell coordinates at the depth limit, [3][n]."""
    mu = np.asarray(means, np.float64)
    X = np.floor((mu - corner[:, None]) / S * float(1 << DEPTH))
    return np.clip(X, 0, (1 << DEPTH) - 1).astype(np.int64)


def tolerance(means, eyes, beta, gamma):
    mu = np.asarray(means, np.float64)
    d = [np.sqrt((mu[0] - e[0]) ** 2 + (mu[1] - e[1]) ** 2 + (mu[2] - e[2]) ** 2) for e in eyes]
    return np.maximum(gamma, beta * np.min(np.array(d), axis=0))


def centre(corner, S, cell, d):
    """Centre of the depth-d cell with integer coordinates `cell` (3 ints)."""
    w = S / float(1 << d)
    return np.array([corner[a] + (cell[a] + 0.5) * w for a in range(3)])


def build_octree(means, eyes, p):
    """Repeated splitting from the root, literally.  Returns (node bytes in depth-first order,
    splat indices in depth-first leaf order, leaf depth per splat, corner, S)."""
    corner, S = root_cube(means)
    X = cells(means, corner, S)
    tol = tolerance(means, eyes, p["beta"], p["gamma"])
    mu = np.asarray(means, np.float64)
    n = mu.shape[1]
    occ = []
    order = []
    dups = []
    depth = np.zeros(n, np.int64)
    leaves = [0]

    def visit(d, cell, members):
        must_split = len(members) > 1
        if not must_split:
            k = members[0]
            c = centre(corner, S, cell, d)
            dist = math.sqrt((mu[0, k] - c[0]) ** 2 + (mu[1, k] - c[1]) ** 2 + (mu[2, k] - c[2]) ** 2)
            must_split = not (dist < tol[k])
        if not must_split or d == DEPTH:
            occ.append(0)  # a leaf
            if len(members) > 1:
                dups.append((leaves[0], len(members) - 1))
            leaves[0] += 1
            for k in sorted(members):
                order.append(k)
                depth[k] = d
            return
        sh = DEPTH - d - 1
        kids = {}
        for k in members:
            cx, cy, cz = ((int(X[a, k]) >> sh) & 1 for a in range(3))
            kids.setdefault(cx << 2 | cy << 1 | cz, []).append(k)
        occ.append(sum(1 << c for c in kids))
        for c in sorted(kids):
            visit(d + 1, (2 * cell[0] + (c >> 2 & 1), 2 * cell[1] + (c >> 1 & 1), 2 * cell[2] + (c & 1)), kids[c])

    visit(0, (0, 0, 0), list(range(n)))
    return bytes(occ), np.array(order, np.int64), depth, corner, S, dups


def quantised_attributes(scene, order, p):
    """Integer attributes in stream order: dict of int64 arrays."""
    ls = np.asarray(scene.log_scales, np.float64)[:, order]
    qt = np.asarray(scene.quats, np.float64)[:, order]
    qn = qt / np.linalg.norm(qt, axis=0, keepdims=True)
    qn = np.where(qn[0] < 0.0, -qn, qn)
    op = 1.0 / (1.0 + np.exp(-np.asarray(scene.opacity_logits, np.float64)[order]))
    sh = np.asarray(scene.sh, np.float64).reshape(48, -1)[:, order]
    out = {"scale": quantise(ls, p["sf_scale"]), "rotation": quantise(qn[1:], p["sf_rotation"]),
           "opacity": quantise(op, p["sf_opacity"])[None, :], "sh": quantise(sh, p["sf_sh"])}
    dc = out["sh"][:3].copy()
    out["sh"][:3] = np.diff(np.concatenate([np.zeros((3, 1), np.int64), dc], axis=1), axis=1)
    return out


def serialise(n, corner, S, p, occ: bytes, dups, attrs: dict) -> bytes:
    head = MAGIC + struct.pack("<II", VERSION, n) + struct.pack("<4d", *corner, S)
    head += struct.pack("<4d", p["sf_scale"], p["sf_rotation"], p["sf_opacity"], p["sf_sh"])
    table = struct.pack("<I", len(dups)) + b"".join(struct.pack("<II", o, c) for o, c in dups)
    body = b"".join(attrs[k].astype("<i4").tobytes() for k in ("scale", "rotation", "opacity", "sh"))
    return head + struct.pack("<I", len(occ)) + occ + table + body


def encode(scene, eyes, q: float = 0.5, p: dict | None = None) -> dict:
    p = p or params(q)
    occ, order, depth, corner, S, dups = build_octree(scene.means, eyes, p)
    attrs = quantised_attributes(scene, order, p)
    raw = serialise(scene.n, corner, S, p, occ, dups, attrs)
    return {"raw": raw, "compressed": zlib.compress(raw, 9), "occupancy": occ, "order": order, "depth": depth,
            "corner": corner, "S": S, "attrs": attrs, "dups": dups}


def decode_positions(occ: bytes, corner, S, dups=()):
    """Leaf centres (one per splat, in stream order) and leaf depths from the node bytes and
    the shared-leaf table."""
    extra = dict(dups)
    out, depths = [], []
    pos = [0]
    leaf = [0]

    def visit(d, cell):
        b = occ[pos[0]]
        pos[0] += 1
        if b == 0:
            for _ in range(1 + extra.get(leaf[0], 0)):
                out.append(centre(corner, S, cell, d))
                depths.append(d)
            leaf[0] += 1
            return
        for c in range(8):
            if b >> c & 1:
                visit(d + 1, (2 * cell[0] + (c >> 2 & 1), 2 * cell[1] + (c >> 1 & 1), 2 * cell[2] + (c & 1)))

    visit(0, (0, 0, 0))
    return np.array(out).T, np.array(depths)


def decode(stream: bytes) -> dict:
    """Inverse of serialise (after zlib): positions, dequantised attributes in stream order."""
    raw = zlib.decompress(stream)
    assert raw[:4] == MAGIC
    version, n = struct.unpack_from("<II", raw, 4)
    c0, c1, c2, S = struct.unpack_from("<4d", raw, 12)
    sf_scale, sf_rot, sf_op, sf_sh = struct.unpack_from("<4d", raw, 44)
    (n_occ,) = struct.unpack_from("<I", raw, 76)
    occ = raw[80:80 + n_occ]
    (n_dup,) = struct.unpack_from("<I", raw, 80 + n_occ)
    dups = [struct.unpack_from("<II", raw, 84 + n_occ + 8 * i) for i in range(n_dup)]
    corner = np.array([c0, c1, c2])
    pos, depths = decode_positions(occ, corner, S, dups)
    body = np.frombuffer(raw[84 + n_occ + 8 * n_dup:], "<i4").astype(np.int64)
    off = 0

    def take(rows):
        nonlocal off
        a = body[off:off + rows * n].reshape(rows, n)
        off += rows * n
        return a

    scale, rot, op, sh = take(3), take(3), take(1), take(48)
    sh = sh.copy()
    sh[:3] = np.cumsum(sh[:3], axis=1)
    xyz = rot / sf_rot
    w = np.sqrt(np.maximum(0.0, 1.0 - (xyz ** 2).sum(axis=0)))
    opacity = (op[0] + 0.25) / sf_op
    oc = np.clip(opacity, 1e-6, 1.0 - 1e-6)
    return {"means": pos, "depths": depths, "log_scales": scale / sf_scale, "quats": np.vstack([w, xyz]),
            "opacity": opacity, "opacity_logits": np.log(oc / (1.0 - oc)), "sh": (sh / sf_sh).reshape(16, 3, n),
            "n_nodes": n_occ, "n_dups": n_dup}
