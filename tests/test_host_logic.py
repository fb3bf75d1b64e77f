"""Host-side logic that needs no GPU: the library's Adam factor table, the bitstream parser, the
camera and image-layout helpers of the compression driver, the autotuner's cache and the buffer
pool that view chunks share."""
import struct
import zlib

import numpy as np
import pytest

from oracle import codec as ocodec


def test_adam_schedule_matches_the_bias_corrections():
    """Row t - 1 of the table holds lr_g / (1 - b1^t) for the six groups and 1 / sqrt(1 - b2^t),
    each rounded once to float from binary64 (Kingma & Ba's bias corrections)."""
    from paper_2601_14821_gb300 import _binding as B
    from paper_2601_14821_gb300 import build

    build.build()
    lr = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)
    b1, b2 = 0.9, 0.999
    tab = B.potr_adam_schedule(1, 600, lr, b1, b2)
    t = np.arange(1, 601, dtype=np.float64)
    b1f, b2f = np.float64(np.float32(b1)), np.float64(np.float32(b2))  # the call takes float32 betas
    for g in range(6):
        want = (np.float64(np.float32(lr[g])) / (1.0 - b1f ** t)).astype(np.float32)
        assert np.array_equal(tab[:, g], want), g
    assert np.array_equal(tab[:, 6], (1.0 / np.sqrt(1.0 - b2f ** t)).astype(np.float32))
    # a later window continues the same table
    assert np.array_equal(B.potr_adam_schedule(101, 5, lr, b1, b2), tab[100:105])
    with pytest.raises(B.PotrError):
        B.potr_adam_schedule(0, 1, lr, b1, b2)


def _oracle_stream(n=40, seed=3):
    import synth

    sc = synth.uniform_cube_scene(n, seed)
    sc.means[:, 7] = sc.means[:, 3]  # a shared depth-limit leaf, so the table is not empty
    eyes = np.array([[3.0, 0.2, 0.0]])
    return ocodec.encode(sc, eyes, p=ocodec.params(0.5))


def test_stream_parser_reads_the_oracle_layout():
    from paper_2601_14821_gb300.codec import parse

    e = _oracle_stream()
    h = parse(e["raw"])
    assert h["n"] == 40 and h["n_nodes"] == len(e["occupancy"]) and h["n_dups"] == len(e["dups"]) >= 1
    a, b = h["nodes"]
    assert e["raw"][a:b] == e["occupancy"]
    a, b = h["dups"]
    assert [tuple(x) for x in np.frombuffer(e["raw"][a:b], "<u4").reshape(-1, 2)] == [tuple(d) for d in e["dups"]]
    a, b = h["attrs"]
    assert (b - a) == 4 * 55 * 40
    want = ocodec.params(0.5)
    for k in ("sf_scale", "sf_rotation", "sf_opacity", "sf_sh"):  # four distinct values, so an order swap shows
        assert h["p"][k] == want[k], k
    np.testing.assert_array_equal(h["cube"], (*e["corner"], e["S"]))


def test_stream_parser_rejects_damaged_streams():
    from paper_2601_14821_gb300.codec import parse

    raw = _oracle_stream()["raw"]
    with pytest.raises(ValueError):
        parse(b"XXXX" + raw[4:])
    with pytest.raises(ValueError):
        parse(raw[:-4])
    assert zlib.decompress(zlib.compress(raw)) == raw
    assert struct.unpack_from("<I", raw, 4)[0] == ocodec.VERSION


def test_camera_centres_recover_the_look_at_positions():
    """The eye of a look-at camera is the position it was built at (the world point the
    world-to-camera map sends to the origin)."""
    import synth
    from paper_2601_14821_gb300.compress import camera_centres

    rng = np.random.default_rng(5)
    pos = rng.normal(0, 3, (7, 3))
    pos[0] = (0.0, 0.0, 4.0)
    cams = [synth.look_at_camera(p, 64 + 8 * i, 48) for i, p in enumerate(pos)]
    got = camera_centres(synth.cameras_to_array(cams))
    assert got.shape == (7, 3) and got.dtype == np.float64
    assert np.allclose(got, pos, rtol=0, atol=1e-5 * (1 + np.abs(pos)))


def test_view_images_follow_the_packed_layout():
    """View v's block starts at 3 * (pixels of views 0..v-1) and holds 3 * width * height floats."""
    import torch

    import synth
    from paper_2601_14821_gb300.compress import view_images

    sizes = [(16, 8), (5, 3), (32, 32)]
    cams = [synth.look_at_camera((0.0, 0.0, 3.0), w, h) for w, h in sizes]
    total = sum(3 * w * h for w, h in sizes)
    buf = torch.arange(total, dtype=torch.float32)
    parts = view_images(synth.cameras_to_array(cams), buf)
    assert [p.numel() for p in parts] == [3 * w * h for w, h in sizes]
    assert torch.equal(torch.cat(parts), buf) and parts[1][0].item() == 3 * 16 * 8


def test_autotune_answers_from_its_cache_file(tmp_path, monkeypatch):
    """The autotuner's key is the GPU model, the splat count rounded down to a power of two and the
    set of view resolutions; a key found in the cache file is answered before any device work."""
    import json

    import torch

    import synth
    from paper_2601_14821_gb300 import batched

    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GPU-under-test")
    monkeypatch.setattr(batched, "_CACHE", {})
    cams = synth.cameras_to_array([synth.look_at_camera((0.0, 0.0, -3.0), 1280, 720),
                                   synth.look_at_camera((1.0, 0.0, -3.0), 640, 480),
                                   synth.look_at_camera((2.0, 0.0, -3.0), 1280, 720)])
    scene = {"means": torch.zeros(3, 3000)}
    key = batched._signature(scene, cams)
    assert key == "GPU-under-test|n~2048|[(640, 480), (1280, 720)]"
    assert batched._signature({"means": torch.zeros(3, 4095)}, cams) == key
    assert batched._signature({"means": torch.zeros(3, 4096)}, cams) != key
    entry = {"tile_w": 8, "tile_h": 32, "batch": 128, "ms_per_view": 1.25, "table": []}
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key: entry}))
    assert batched.autotune(scene, cams, device="cpu", cache_path=str(path)) == entry


def test_buffer_pool_shares_and_grows_named_buffers():
    """A name is one buffer: typed views of it share storage, a larger request replaces it, a
    smaller one reuses it, and every view starts 16-byte aligned (potr_preprocess rejects raster
    and culling arrays that are not)."""
    import torch

    from paper_2601_14821_gb300.pipeline import BufferPool

    pool = BufferPool("cpu")
    a = pool.get("raster", 12, torch.float32)
    b = pool.get("raster", 6, torch.int64)
    assert a.numel() == 12 and b.numel() == 6 and a.data_ptr() == b.data_ptr()
    big = pool.get("raster", 1000, torch.float32)
    assert big.numel() == 1000 and pool.nbytes() == 4000
    small = pool.get("raster", 3, torch.int32)
    assert small.data_ptr() == big.data_ptr()
    other = pool.get("cull", 0, torch.int32)  # at least one element
    assert other.numel() == 1 and pool.nbytes() == 4004
    for t in (a, big, other):
        assert t.data_ptr() % 16 == 0
