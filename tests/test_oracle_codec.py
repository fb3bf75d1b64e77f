"""Pins of the codec oracle (Section IV-E) against facts fixed outside it."""
import math

import numpy as np

import synth
from oracle import codec


def test_quantiser_rounds_half_up():
    x = np.array([0.0, 0.49, 0.5, -0.5, -0.51, 1.5, 2.4999]) / 10.0
    assert list(codec.quantise(x, 10.0)) == [0, 0, 1, 0, -1, 2, 2]


def test_two_splats_hand_worked_stream():
    """Splats at opposite corners of the unit cube, one eye 1000 away: tolerance 1.4e-4 q x 1000
    = 0.07 (q = 0.5), so each ends in the corner cell of depth 4 (centre sqrt(3)/2^5 = 0.054 away;
    depth 3 gives 0.108).  Root: children 0 and 7 (0x81); then three single-child nodes (0x01 or
    0x80) and a leaf (0x00) per splat."""
    means = np.array([[0.0, 1.0], [0.0, 1.0], [0.0, 1.0]], np.float32)
    eyes = [np.array([0.5, 0.5, 1000.0])]
    p = codec.params(0.5)
    occ, order, depth, corner, S, dups = codec.build_octree(means, eyes, p)
    assert not dups and occ == bytes([0x81, 0x01, 0x01, 0x01, 0x00, 0x80, 0x80, 0x80, 0x00])
    assert list(order) == [0, 1] and list(depth) == [4, 4]
    pos, dep = codec.decode_positions(occ, corner, S)
    np.testing.assert_allclose(pos[:, 0], [1 / 32] * 3)
    np.testing.assert_allclose(pos[:, 1], [1 - 1 / 32] * 3)


def test_coincident_splats_share_a_depth_limit_leaf_listed_in_the_table():
    """Splats 0 and 1 coincide at the cube's corner (0,0,0), splat 2 sits at (1,1,1): the root has
    children 0 and 7; splats 0 and 1 split down to depth 21 (20 single-child bytes 0x01, then a
    leaf), and that leaf -- the first in depth-first order -- holds one extra splat, so the table
    reads (0, 1); splat 2 ends at depth 4 as in the two-splat stream.  The serialised stream
    carries the node count, the nodes, the table size and the pair, little-endian."""
    means = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0], [0.0, 0.0, 1.0]], np.float32)
    eyes = [np.array([0.5, 0.5, 1000.0])]
    p = codec.params(0.5)
    occ, order, depth, corner, S, dups = codec.build_octree(means, eyes, p)
    want = bytes([0x81] + [0x01] * 20 + [0x00] + [0x80] * 3 + [0x00])
    assert occ == want and dups == [(0, 1)]
    assert list(order) == [0, 1, 2] and list(depth) == [21, 21, 4]
    pos, dep = codec.decode_positions(occ, corner, S, dups)
    np.testing.assert_allclose(pos[:, 0], [0.5 / 2 ** 21] * 3)
    np.testing.assert_allclose(pos[:, 1], pos[:, 0])
    np.testing.assert_allclose(pos[:, 2], [1 - 1 / 32] * 3)
    assert list(dep) == [21, 21, 4]

    class Sc:
        n = 3
    sc = Sc()
    sc.means = means
    sc.log_scales = np.zeros((3, 3), np.float32)
    sc.quats = np.tile(np.array([[1.0], [0.0], [0.0], [0.0]], np.float32), (1, 3))
    sc.opacity_logits = np.zeros(3, np.float32)
    sc.sh = np.zeros((16, 3, 3), np.float32)
    raw = codec.encode(sc, eyes, p=p)["raw"]
    assert raw[76:80] == (len(want)).to_bytes(4, "little") and raw[80:80 + len(want)] == want
    assert raw[80 + len(want):80 + len(want) + 12] == bytes([1, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0])
    assert len(raw) == 80 + len(want) + 12 + 4 * 55 * 3


def test_round_trip_honours_the_precision_criterion_and_the_quantisers():
    sc = synth.uniform_cube_scene(3000, 9)
    eyes = [np.array([3.0, 0.2, 0.0]), np.array([-2.0, 0.0, 2.5]), np.array([0.0, 3.0, -0.5])]
    p = codec.params(0.5)
    e = codec.encode(sc, eyes, p=p)
    d = codec.decode(e["compressed"])
    o = e["order"]
    mu = sc.means[:, o].astype(np.float64)
    tol = codec.tolerance(mu, eyes, p["beta"], p["gamma"])
    err = np.linalg.norm(d["means"] - mu, axis=0)
    assert np.all(err < tol) and np.array_equal(d["depths"], e["depth"][o])
    assert np.max(np.abs(d["log_scales"] - sc.log_scales[:, o])) <= 0.5 / p["sf_scale"] + 1e-12
    assert np.max(np.abs(d["sh"] - sc.sh[:, :, o])) <= 0.5 / p["sf_sh"] + 1e-9
    op = 1.0 / (1.0 + np.exp(-sc.opacity_logits[o].astype(np.float64)))
    assert np.max(np.abs(d["opacity"] - op)) <= 0.75 / p["sf_opacity"] + 1e-12
    sig = 1.0 / (1.0 + np.exp(-d["opacity_logits"]))
    assert np.max(np.abs(sig - np.clip(d["opacity"], 1e-6, 1 - 1e-6))) < 1e-12
    q = sc.quats[:, o].astype(np.float64)
    q = q / np.linalg.norm(q, axis=0)
    q = np.where(q[0] < 0, -q, q)
    assert np.max(np.abs(d["quats"][1:] - q[1:])) <= 0.5 / p["sf_rotation"] + 1e-12
    # the real part is rebuilt so that the quaternion has unit norm (where |xyz~| <= 1), and it
    # is within sqrt(|w~^2 - w^2|) <= sqrt(2 delta + 3 delta^2) of the original, delta = the
    # norm of the xyz rounding error
    xyz = d["quats"][1:]
    inside = (xyz ** 2).sum(axis=0) <= 1.0
    assert inside.mean() > 0.9 and np.all(d["quats"][0, ~inside] == 0.0)  # rounding past 1: w = 0
    assert np.max(np.abs(np.linalg.norm(d["quats"][:, inside], axis=0) - 1.0)) < 1e-12
    delta = math.sqrt(3.0) * 0.5 / p["sf_rotation"]
    assert np.max(np.abs(d["quats"][0] - q[0])) <= math.sqrt(2.0 * delta + 3.0 * delta * delta)
    assert len(e["compressed"]) < len(e["raw"])


def test_nearest_eye_sets_the_tolerance():
    """The precision criterion takes the distance to the nearest eye: an eye farther from every
    splat than the others changes no byte of the stream, and an eye among the splats refines the
    octree."""
    sc = synth.uniform_cube_scene(2000, 12)
    eyes = [np.array([3.0, 0.2, 0.0]), np.array([-2.0, 0.0, 2.5])]
    p = codec.params(0.5)
    base = codec.encode(sc, eyes, p=p)
    far = codec.encode(sc, eyes + [np.array([60.0, -45.0, 80.0])], p=p)
    assert far["raw"] == base["raw"]
    near = codec.encode(sc, eyes + [sc.means.astype(np.float64).mean(axis=1)], p=p)
    assert len(near["occupancy"]) > len(base["occupancy"])


def _sorted_formulation(means, eyes, p):
    """The same octree from the splats sorted by cell code: a splat's leaf is the first depth at
    or below the point where its cell holds no other splat (one more than the longest common
    cell prefix with its neighbours) that passes the precision test."""
    corner, S = codec.root_cube(means)
    X = codec.cells(means, corner, S)
    n = X.shape[1]
    code = np.zeros(n, dtype=object)
    for k in range(n):
        c = 0
        for b in range(codec.DEPTH - 1, -1, -1):
            c = (c << 3) | ((int(X[0, k]) >> b & 1) << 2) | ((int(X[1, k]) >> b & 1) << 1) | (int(X[2, k]) >> b & 1)
        code[k] = c
    order = sorted(range(n), key=lambda k: (code[k], k))

    def lcp(a, b):
        for d in range(codec.DEPTH):
            s = 3 * (codec.DEPTH - 1 - d)
            if (a >> s) != (b >> s):
                return d
        return codec.DEPTH

    tol = codec.tolerance(means, eyes, p["beta"], p["gamma"])
    mu = np.asarray(means, np.float64)
    depth = np.zeros(n, np.int64)
    for i, k in enumerate(order):
        l = max(lcp(code[order[i - 1]], code[k]) if i > 0 else -1,
                lcp(code[order[i + 1]], code[k]) if i + 1 < n else -1)
        d = min(l + 1, codec.DEPTH)
        while d < codec.DEPTH:
            cell = [int(X[a, k]) >> (codec.DEPTH - d) for a in range(3)]
            c = codec.centre(corner, S, cell, d)
            if math.sqrt((mu[0, k] - c[0]) ** 2 + (mu[1, k] - c[1]) ** 2 + (mu[2, k] - c[2]) ** 2) < tol[k]:
                break
            d += 1
        depth[k] = d
    return np.array(order), depth


def test_splitting_equals_the_sorted_formulation():
    rng = np.random.default_rng(2)
    eyes = [np.array([2.0, 0.1, 0.3]), np.array([0.0, -2.5, 1.0])]
    p = codec.params(0.7)
    for n in (1, 2, 17, 400):
        means = rng.uniform(-1, 1, (3, n)).astype(np.float32)
        if n > 10:
            means[:, 5] = means[:, 3]  # two splats in one cell: split to the depth limit
        occ, order, depth, corner, S, dups = codec.build_octree(means, eyes, p)
        o2, d2 = _sorted_formulation(means, eyes, p)
        assert np.array_equal(order, o2) and np.array_equal(depth, d2), n
        if n > 10:
            assert depth[5] == codec.DEPTH and depth[3] == codec.DEPTH and len(dups) == 1 and dups[0][1] == 1
            pos, dep = codec.decode_positions(occ, corner, S, dups)
            assert pos.shape[1] == n


def _parallel_parse(occ: bytes, corner, S, dups):
    """Leaf centres from the node bytes without recursion: e_i = sum_{j<i} (c_j - 1) (c_j the
    children of node j) counts the pending subtrees when node i is met; node i's parent is the
    last j < i with e_j <= e_i, and it is that parent's child number e_j + c_j - 1 - e_i."""
    c = [bin(b).count("1") for b in occ]
    e = np.concatenate([[0], np.cumsum(np.array(c) - 1)])
    assert e[-1] == -1 and np.all(e[:-1] >= 0)
    m = len(occ)
    par, octant = [0] * m, [0] * m
    for i in range(1, m):
        j = max(j for j in range(i) if e[j] <= e[i])
        r = e[j] + c[j] - 1 - e[i]
        bits = [k for k in range(8) if occ[j] >> k & 1]
        par[i], octant[i] = j, bits[r]
    extra = dict(dups)
    out, ordinal = [], 0
    for i in range(m):
        if occ[i]:
            continue
        cell, d, k = [0, 0, 0], 0, i
        while k:
            o = octant[k]
            cell = [cell[0] | (o >> 2 & 1) << d, cell[1] | (o >> 1 & 1) << d, cell[2] | (o & 1) << d]
            d += 1
            k = par[k]
        out += [codec.centre(corner, S, cell, d)] * (1 + extra.get(ordinal, 0))
        ordinal += 1
    return np.array(out).T


def test_parallel_parse_formulation_equals_the_recursive_decode():
    rng = np.random.default_rng(5)
    eyes = [np.array([2.0, 0.1, 0.3])]
    for n, q in ((1, 0.5), (2, 0.5), (40, 0.2), (300, 0.9)):
        means = rng.uniform(-1, 1, (3, n)).astype(np.float32)
        if n > 10:
            means[:, 9] = means[:, 4]
            means[:, 21] = means[:, 4]
            means[:, 30] = means[:, 12]
        occ, order, depth, corner, S, dups = codec.build_octree(means, eyes, codec.params(q))
        want, _ = codec.decode_positions(occ, corner, S, dups)
        got = _parallel_parse(occ, corner, S, dups)
        assert np.array_equal(got, want), n


def test_single_splat_closed_form():
    """One splat: the root cube has its corner at the splat and edge 1, so the splat lies at the
    corner of every cell on its path (child 0 each time) and its leaf is the first depth d at
    which the cell centre, 0.5 sqrt(3) 2^-d away, is within the tolerance max(gamma, beta |mu - eye|)."""
    sc = synth.uniform_cube_scene(1, 3)
    eye = np.array([3.0, 0.2, 0.0])
    p = codec.params(0.5)
    mu = sc.means[:, 0].astype(np.float64)
    tol = max(p["gamma"], p["beta"] * float(np.linalg.norm(mu - eye)))
    d = next(k for k in range(codec.DEPTH + 1) if 0.5 * math.sqrt(3.0) * 2.0 ** -k < tol)
    e = codec.encode(sc, [eye], p=p)
    assert e["S"] == 1.0 and np.array_equal(e["corner"], mu)
    assert e["occupancy"] == bytes([1] * d + [0]) and e["depth"].tolist() == [d]
    dec = codec.decode(e["compressed"])
    np.testing.assert_allclose(dec["means"][:, 0], mu + 0.5 * 2.0 ** -d, rtol=0, atol=1e-15)
