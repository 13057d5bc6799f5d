"""Frame-sharded fusion (host logic of paper_2111_11103_gb300.shard) on CPU
ranks: frame ranges partition the sequence, and the all-reduced state of two
gloo ranks that each fused half of the frames (with the oracle) equals the
one-rank fusion of the whole sequence."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import scenegen as sg
from paper_2111_11103_gb300.shard import allreduce_state, frame_range


@pytest.mark.parametrize("n", [0, 1, 7, 8, 1000])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_frame_ranges_partition(n, world):
    seen = []
    for r in range(world):
        a, b = frame_range(n, r, world)
        assert 0 <= a <= b <= n
        assert b - a in (n // world, n // world + 1)
        seen.extend(range(a, b))
    assert seen == list(range(n))


def test_frame_range_rejects_bad_shards():
    for args in [(5, 2, 2), (5, -1, 2), (5, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            frame_range(*args)


def test_allreduce_state_checks_types():
    with pytest.raises(TypeError):
        allreduce_state(torch.zeros(2, 3, dtype=torch.float64), torch.zeros(2, dtype=torch.int32))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, rule, weight, out_dir):
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        scene, cams = sg.tiny_room(), sg.circle_poses()
        probs = sg.predictions(scene, cams, "tiny", device="cpu").numpy()
        mesh = oracle.Mesh(scene.vertices, scene.faces)
        a, b = frame_range(cams.K.shape[0], rank, world)
        A, cnt = oracle.fuse_sequence(mesh, cams.K[a:b], cams.cam_to_world[a:b], probs[a:b], rule, weight)
        acc = torch.as_tensor(A.astype(np.float32))
        c = torch.as_tensor(cnt.astype(np.int32))
        allreduce_state(acc, c)
        np.save(os.path.join(out_dir, f"acc{rank}.npy"), acc.numpy())
        np.save(os.path.join(out_dir, f"cnt{rank}.npy"), c.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("rule,weight", [("logsum", "pixel"), ("sum", "image")])
def test_two_gloo_ranks_match_one_rank(ora, tmp_path, rule, weight):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), rule, weight, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    scene, cams = sg.tiny_room(), sg.circle_poses()
    probs = sg.predictions(scene, cams, "tiny", device="cpu").numpy()
    A, cnt = ora.fuse_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world, probs, rule, weight)
    for r in range(world):
        acc = np.load(tmp_path / f"acc{r}.npy").astype(np.float64)
        c = np.load(tmp_path / f"cnt{r}.npy")
        assert np.array_equal(c, cnt)
        # float32 sum of two float32-rounded halves against the binary64 whole
        np.testing.assert_allclose(acc, A, rtol=1e-6, atol=1e-6 * np.abs(A).max())
