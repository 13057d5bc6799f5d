"""Failure detection without a GPU fault.

* A bounded wait that runs out: the test hook LABELFUSE_TEST_SKIP_TILE makes
  the scatter's producer leave one pipeline stage unfilled, so the consumers'
  waits on it give up after their (shortened) limit instead of spinning.  The
  kernel returns, sm_check reports SM_ERR_TIMEOUT, and the next call on the
  same GPU fuses correctly (against the oracle).
* Device allocations that fail: with LABELFUSE_TEST_FAIL_ALLOC set every
  allocation of the library reports out-of-memory (host-side injection, no
  memory is exhausted).  The calls return SM_ERR_OOM, a mesh that was already
  uploaded stays usable, and once the variable is unset the same calls
  succeed and match the oracle.
"""
import os

import numpy as np
import pytest
import torch

import scenegen as sg
from gpu_common import assert_acc_close, to_dev

pytestmark = pytest.mark.gpu

SM_ERR_OOM = 2
SM_ERR_TIMEOUT = 5


@pytest.fixture()
def tiny():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    dev = torch.device("cuda:0")
    scene, cams = sg.tiny_room(), sg.circle_poses()
    return dev, scene, cams, sg.predictions(scene, cams, "tiny", device=dev)


def _fuse_and_compare(ora, lf, m, dev, scene, cams, probs, rule, weight):
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    _, _, K, T, _ = to_dev(scene, cams, None, dev)
    idm = torch.empty((N, H, W), dtype=torch.int32, device=dev)
    lf.sm_reset(m)
    lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W, idm)
    n_x = lf.sm_num_rows(m)
    acc = torch.empty((n_x, c), device=dev)
    cnt = torch.empty(n_x, dtype=torch.int32, device=dev)
    lf.sm_read_state(m, acc, cnt)
    lf.sm_check(m)
    A, cnt_o, idm_o = ora.fuse_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world,
                                        probs.cpu().numpy(), rule, weight, want_idmaps=True)
    assert np.array_equal(idm.cpu().numpy(), idm_o)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), cnt_o)
    assert_acc_close(acc.cpu().numpy(), A)


@pytest.fixture()
def room20():
    """A small paper-shaped room with c = 20: pixel weights fuse through the
    persistent work-queue kernel."""
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    dev = torch.device("cuda:0")
    scene = sg.paper_room(target_faces=20_000, n_classes=20)
    cams = sg.random_walk_poses(8, H=96, W=128, fx=115.0, fy=115.0, cx=63.5, cy=47.5)
    return dev, scene, cams, sg.predictions(scene, cams, "paper", device=dev)


@pytest.mark.parametrize("case,weight", [("tiny", "pixel"), ("tiny", "image"), ("room20", "pixel")])
def test_scatter_wait_runs_out_and_recovers(ora, request, monkeypatch, case, weight):
    """Stream-ordered scatter (c = 4, both weights) and the work-queue kernel
    (c = 20, pixel weights): a stage that is never filled makes the waits give
    up; the call is reported as SM_ERR_TIMEOUT and the next one is exact."""
    from paper_2111_11103_gb300 import labelfuse as lf
    dev, scene, cams, probs = request.getfixturevalue(case)
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "logsum", weight)
    try:
        if case == "room20":
            lf.sm_set_queue_shape(m, H, W, 4, 1, 1, 16)
        monkeypatch.setenv("LABELFUSE_TEST_SKIP_TILE", "0")
        lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W)   # enqueued fine; the kernel gives up
        with pytest.raises(lf.LabelFuseError) as ei:
            lf.sm_check(m)
        assert ei.value.status == SM_ERR_TIMEOUT
        lf.sm_check(m)  # the latch was cleared by the read
        monkeypatch.delenv("LABELFUSE_TEST_SKIP_TILE")
        _fuse_and_compare(ora, lf, m, dev, scene, cams, probs, "logsum", weight)
    finally:
        lf.sm_mesh_free(m)


def test_allocation_failures_return_oom_and_leave_the_mesh_usable(ora, tiny, monkeypatch):
    from paper_2111_11103_gb300 import labelfuse as lf
    dev, scene, cams, probs = tiny
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "sum", "image")
    try:
        monkeypatch.setenv("LABELFUSE_TEST_FAIL_ALLOC", "1")
        with pytest.raises(lf.LabelFuseError) as ei:   # upload: the first allocation fails
            lf.sm_mesh_upload(V, Fc, None, c, "sum", "pixel")
        assert ei.value.status == SM_ERR_OOM
        with pytest.raises(lf.LabelFuseError) as ei:   # fusion: the scratch cannot grow
            lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W)
        assert ei.value.status == SM_ERR_OOM
        h_img = torch.empty((N, H, W), dtype=torch.uint8)
        with pytest.raises(lf.LabelFuseError) as ei:   # host streaming: no staging
            lf.sm_fuse_render_host(m, probs.cpu(), "f32", None, K.cpu(), T.cpu(), N, H, W, h_img)
        assert ei.value.status == SM_ERR_OOM
        monkeypatch.delenv("LABELFUSE_TEST_FAIL_ALLOC")
        lf.sm_check(m)
        _fuse_and_compare(ora, lf, m, dev, scene, cams, probs, "sum", "image")
    finally:
        lf.sm_mesh_free(m)
    assert "LABELFUSE_TEST_FAIL_ALLOC" not in os.environ
