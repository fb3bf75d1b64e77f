"""Multi-rank host logic on CPU: world_size 2 over gloo (127.0.0.1), no GPU.

Covers the view sharding, the max-over-ranks timing reduction and the deterministic rank-order
sum that combines per-rank dMSE partials; the sharded oracle result must equal the
single-process one.
"""
import os
import socket

import numpy as np
import torch
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import oracle
    import synth
    from paper_2601_14821_gb300 import dist as D

    D.init("gloo")
    assert D.active()
    assert D.max_over_ranks(float(rank + 1)) == float(world)
    assert D.sum_over_ranks(1.0) == float(world)
    # shard 3 views of the tiny scene over the ranks and combine the dMSE partials
    sc = synth.uniform_cube_scene(600, 21)
    cams = [synth.look_at_camera((0, 0, -3), 64, 48), synth.look_at_camera((2, 0.5, -2), 48, 64),
            synth.look_at_camera((-3, 0, 0.5), 64, 64)]
    cfg = oracle.make_config()
    targets = [np.full((3, c.height, c.width), 0.2, np.float32) for c in cams]
    s, e = D.shard_range(len(cams), rank, world)
    act = oracle.activate(sc)
    local = np.zeros(sc.n)
    for v in range(s, e):
        d, _ = oracle.view_dsse(sc, cams[v], cfg, targets[v], act)
        local += d / (3.0 * cams[v].pixels) / len(cams)
    total = D.ordered_sum(torch.from_numpy(local)).numpy()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), total)
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_shard_range_partitions():
    from paper_2601_14821_gb300.dist import shard_range

    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_gloo_sharded_dmse(tmp_path):
    import oracle
    import synth

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert np.array_equal(r0, r1)  # every rank holds the same bits
    sc = synth.uniform_cube_scene(600, 21)
    cams = [synth.look_at_camera((0, 0, -3), 64, 48), synth.look_at_camera((2, 0.5, -2), 48, 64),
            synth.look_at_camera((-3, 0, 0.5), 64, 64)]
    want, _ = oracle.dmse(sc, cams, oracle.make_config(), [np.full((3, c.height, c.width), 0.2, np.float32) for c in cams])
    np.testing.assert_allclose(r0, want, rtol=1e-13, atol=1e-18)
    assert np.count_nonzero(want) > 100
