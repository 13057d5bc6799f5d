"""Launch-side features: a whole fusion step captured into a CUDA graph and
replayed, the frames-per-launch autotuner, and independent scenes fused side
by side on several streams -- each against the oracle."""
import numpy as np
import pytest
import torch

import scenegen as sg
from gpu_common import GpuResult, assert_acc_close, check_against_oracle, run_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2111_11103_gb300 import labelfuse as lf
    lf.lib()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def medium(dev):
    scene = sg.paper_room(target_faces=60_000)
    cams = sg.random_walk_poses(24, H=151, W=203, fx=183.0, fy=183.0, cx=101.0, cy=75.0)
    return scene, cams, sg.predictions(scene, cams, "paper", device=dev)


def _state(lf, m, n_x, c, dev):
    acc = torch.empty((n_x, c), device=dev)
    cnt = torch.empty(n_x, dtype=torch.int32, device=dev)
    lf.sm_read_state(m, acc, cnt)
    return acc.cpu().numpy(), cnt.cpu().numpy()


def test_step_captured_in_a_cuda_graph(ora, dev, medium):
    """A whole step (reset, fuse, normalise, render-back) captured once and
    replayed three times: row maps, counts, accumulators, labels and label
    images against the oracle after the last replay."""
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "logsum", "pixel")
    try:
        n_x = lf.sm_num_rows(m)
        idm = torch.empty((N, H, W), dtype=torch.int32, device=dev)
        img = torch.empty((N, H, W), dtype=torch.uint8, device=dev)
        labels = torch.empty(n_x, dtype=torch.int32, device=dev)
        dist = torch.empty((n_x, c), dtype=torch.float32, device=dev)

        def step():
            lf.sm_reset(m)
            lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W, idm)
            lf.sm_normalise(m, dist, labels)
            lf.sm_render_idmap(m, idm, N * H * W, img)

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            step()  # eager: grows the scratch to this size
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(3):
            idm.fill_(-9)
            img.fill_(7)
            labels.fill_(-5)
            g.replay()
        torch.cuda.synchronize()
        lf.sm_check(m)
        acc1, cnt1 = _state(lf, m, n_x, c, dev)
    finally:
        lf.sm_mesh_free(m)
    res = GpuResult(idm.cpu().numpy(), acc1, cnt1.astype(np.int64), dist.cpu().numpy(), labels.cpu().numpy(),
                    img.cpu().numpy(), None, n_x)
    check_against_oracle(ora, scene, cams, probs.cpu().numpy(), res, "logsum", "pixel", nthreads=8)


def test_autotuner_picks_a_batch_and_keeps_results(ora, dev, medium):
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "sum", "pixel")
    try:
        best = lf.sm_autotune_batch(m, probs, "f32", None, K, T, N, H, W)
        assert best % 4 == 0 and 4 <= best <= N
        acc, cnt = _state(lf, m, lf.sm_num_rows(m), c, dev)
        assert float(np.abs(acc).max()) == 0.0 and int(cnt.max()) == 0  # reset afterwards
        lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W)
        acc, cnt = _state(lf, m, lf.sm_num_rows(m), c, dev)
        lf.sm_check(m)
        with pytest.raises(lf.LabelFuseError):
            lf.sm_autotune_batch(m, probs, "f32", None, K, T, 3, H, W)
    finally:
        lf.sm_mesh_free(m)
    A, cnt_o = ora.fuse_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world,
                                 probs.cpu().numpy(), "sum", "pixel", nthreads=8)
    assert np.array_equal(cnt.astype(np.int64), cnt_o)
    assert_acc_close(acc, A)


def test_scenes_side_by_side_match_the_oracle(ora, dev):
    """Four scenes of different size, resolution and class count fused side by
    side on three streams, eagerly and as one captured CUDA graph: each
    scene's counts and accumulators against the oracle."""
    from paper_2111_11103_gb300 import labelfuse as lf
    from paper_2111_11103_gb300.scenes import SceneJob, fuse_scenes
    specs = [(sg.tiny_room(), sg.circle_poses(n=6)),
             (sg.paper_room(target_faces=20_000), sg.random_walk_poses(10, H=96, W=128, fx=115.0, fy=115.0,
                                                                         cx=63.5, cy=47.5)),
             (sg.paper_room(seed=77, target_faces=30_000, n_classes=20),
              sg.random_walk_poses(7, seed=9, H=120, W=160, fx=150.0, fy=150.0, cx=79.5, cy=59.5)),
             (sg.tiny_room(), sg.circle_poses(n=5, H=40, W=52, fx=45.0, fy=45.0, cx=26.0, cy=20.0))]
    jobs, expect, meshes = [], [], []
    try:
        for scene, cams in specs:
            probs = sg.predictions(scene, cams, "tiny" if scene.n_classes == 4 else "paper", device=dev)
            expect.append(ora.fuse_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world,
                                            probs.cpu().numpy(), "logsum", "image", nthreads=8))
            V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
            m = lf.sm_mesh_upload(V, Fc, None, scene.n_classes, "logsum", "image")
            meshes.append(m)
            jobs.append(SceneJob(m, probs, K, T, cams.H, cams.W,
                                 labels_out=torch.empty(lf.sm_num_rows(m), dtype=torch.int32, device=dev)))

        def check():
            for j, (A, cnt_o), (scene, _) in zip(jobs, expect, specs):
                acc, cnt = _state(lf, j.mesh, lf.sm_num_rows(j.mesh), scene.n_classes, dev)
                lf.sm_check(j.mesh)
                assert np.array_equal(cnt.astype(np.int64), cnt_o)
                assert_acc_close(acc, A)

        fuse_scenes(jobs, streams=3)
        torch.cuda.synchronize()
        check()
        with pytest.raises(ValueError):
            fuse_scenes([jobs[0], jobs[0]])
        # the same multi-stream submission captured into one CUDA graph and replayed
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for j in jobs:
                lf.sm_reset(j.mesh)
            fuse_scenes(jobs, streams=3)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        check()
    finally:
        for m in meshes:
            lf.sm_mesh_free(m)


def test_fuse_scenes_work_queue_matches_the_oracle(ora, dev):
    """sm_fuse_scenes on an uneven batch: scenes with c = 20 and 40, F32 and
    BF16 storage, 5-13 frames of different sizes and different queue shapes
    share persistent work-queue launches (grouped by class count, storage
    type and rule); a c = 4 scene and a texel-mode scene take the per-scene
    path.  Every scene's row maps, counts and accumulators against the
    oracle, on two calls in a row."""
    from paper_2111_11103_gb300 import labelfuse as lf
    from test_gpu_parity import _quantise
    specs = [  # (scene, cams, dtype, texel steps, queue shape or None)
        (sg.paper_room(seed=11, target_faces=20_000, n_classes=20),
         sg.random_walk_poses(7, seed=3, H=120, W=160, fx=150.0, fy=150.0, cx=79.5, cy=59.5), "f32", None,
         (4, 1, 1, 16)),
        (sg.paper_room(seed=12, target_faces=30_000), sg.random_walk_poses(13, seed=4, H=96, W=128, fx=115.0,
                                                                            fy=115.0, cx=63.5, cy=47.5),
         "f32", None, (8, 2, 2, 64)),
        (sg.paper_room(seed=13, target_faces=15_000), sg.random_walk_poses(5, seed=5, H=151, W=203, fx=183.0,
                                                                            fy=183.0, cx=101.0, cy=75.0),
         "bf16", None, None),
        (sg.paper_room(seed=14, target_faces=25_000, n_classes=20),
         sg.random_walk_poses(9, seed=6, H=48, W=64, fx=58.0, fy=58.0, cx=31.5, cy=23.5), "f32", None, (4, 3, 1, 1)),
        (sg.tiny_room(), sg.circle_poses(n=6), "f32", None, None),
        (sg.paper_room(seed=15, target_faces=10_000, n_classes=20),
         sg.random_walk_poses(6, seed=7, H=64, W=96, fx=80.0, fy=80.0, cx=47.5, cy=31.5), "f32", 2, None),
    ]
    meshes, calls, checks = [], [], []
    try:
        for scene, cams, dtype, texel, shape in specs:
            N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
            probs = sg.predictions(scene, cams, "tiny" if c == 4 else "paper", device=dev)
            if dtype == "f32":
                q, scale, deq = probs, None, probs.cpu().numpy()
            else:
                q, scale, deq = _quantise(probs, dtype)
            s = None if texel is None else np.full(len(scene.faces), texel, dtype=np.int32)
            V, Fc, K, T, tr = to_dev(scene, cams, s, dev)
            m = lf.sm_mesh_upload(V, Fc, tr, c, "logsum", "pixel")
            meshes.append(m)
            if shape is not None:
                lf.sm_set_queue_shape(m, H, W, *shape)
            idm = torch.full((N, H, W), -9, dtype=torch.int32, device=dev)
            calls.append((m, q, dtype, scale, K, T, N, H, W, idm))
            A, cnt, idm_o = ora.fuse_sequence(ora.Mesh(scene.vertices, scene.faces, texel_res=s), cams.K,
                                              cams.cam_to_world, deq, "logsum", "pixel", nthreads=8, want_idmaps=True)
            checks.append((m, c, idm, A, cnt, idm_o))
        for _ in range(2):
            for m in meshes:
                lf.sm_reset(m)
            lf.sm_fuse_scenes(calls)
            torch.cuda.synchronize()
            for m, c, idm, A, cnt_o, idm_o in checks:
                acc, cnt = _state(lf, m, lf.sm_num_rows(m), c, dev)
                lf.sm_check(m)
                assert np.array_equal(idm.cpu().numpy(), idm_o)
                assert np.array_equal(cnt.astype(np.int64), cnt_o)
                assert_acc_close(acc, A)
        with pytest.raises(lf.LabelFuseError):
            lf.sm_fuse_scenes([calls[0], calls[0]])
    finally:
        for m in meshes:
            lf.sm_mesh_free(m)
