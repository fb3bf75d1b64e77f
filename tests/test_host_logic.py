"""Host-side logic that needs no GPU: the library's Adam factor table and the bitstream parser."""
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
    assert h["p"]["sf_sh"] == ocodec.params(0.5)["sf_sh"]
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
