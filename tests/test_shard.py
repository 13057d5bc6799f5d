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


class _FakeMesh:
    """Stands in for a library mesh on a CPU rank: the state that
    sm_read_state / sm_load_state would copy out of and into the device."""

    def __init__(self, acc, cnt):
        self.acc, self.cnt = acc, cnt


def _complete_main(rank, world, port, out_dir):
    """One CPU rank runs shard.complete_fusion (the library's sharded
    completion step) with the library's state calls replaced by fakes over an
    oracle-fused half of the frames."""
    import oracle
    from paper_2111_11103_gb300 import labelfuse as lf
    from paper_2111_11103_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        scene, cams = sg.tiny_room(), sg.circle_poses()
        probs = sg.predictions(scene, cams, "tiny", device="cpu").numpy()
        mesh = oracle.Mesh(scene.vertices, scene.faces)
        a, b = frame_range(cams.K.shape[0], rank, world)
        A, cnt = oracle.fuse_sequence(mesh, cams.K[a:b], cams.cam_to_world[a:b], probs[a:b], "sum", "pixel")
        fake = _FakeMesh(torch.as_tensor(A.astype(np.float32)), torch.as_tensor(cnt.astype(np.int32)))
        handles = {1: fake}
        lf.sm_num_rows = lambda m: handles[m].acc.shape[0]
        lf.sm_num_classes = lambda m: handles[m].acc.shape[1]

        def read(m, acc, cnt, stream=None):
            acc.copy_(handles[m].acc)
            cnt.copy_(handles[m].cnt)

        def load(m, acc, cnt, stream=None):
            handles[m].acc, handles[m].cnt = acc.clone(), cnt.clone()

        lf.sm_read_state, lf.sm_load_state = read, load
        state = (torch.empty_like(fake.acc), torch.empty_like(fake.cnt))
        shard.complete_fusion(1, state)
        np.save(os.path.join(out_dir, f"acc{rank}.npy"), handles[1].acc.numpy())
        np.save(os.path.join(out_dir, f"cnt{rank}.npy"), handles[1].cnt.numpy())
    finally:
        dist.destroy_process_group()


def test_complete_fusion_over_two_gloo_ranks(ora, tmp_path):
    """The sharded completion step of the library's host path (read state,
    all-reduce, load state) on two CPU ranks: each rank ends with the whole
    sequence's counts and accumulators."""
    world = 2
    mp.start_processes(_complete_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    scene, cams = sg.tiny_room(), sg.circle_poses()
    probs = sg.predictions(scene, cams, "tiny", device="cpu").numpy()
    A, cnt = ora.fuse_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world, probs, "sum",
                               "pixel")
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"cnt{r}.npy"), cnt)
        np.testing.assert_allclose(np.load(tmp_path / f"acc{r}.npy").astype(np.float64), A, rtol=1e-6,
                                   atol=1e-6 * np.abs(A).max())
