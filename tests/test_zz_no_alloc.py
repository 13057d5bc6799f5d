"""The allocation-free entry point sm_render_rows_noalloc.

It serves callers that cannot allocate device memory (a plugin whose host
application owns all device memory through its own pool, or a latency-bound
loop that must not call cudaMalloc, which can block and synchronise the
device).  It renders row maps with the library's static scratch instead.  Its
output must equal the row maps of the allocating entry point sm_fuse_frames
bit for bit, on two calls in a row (the second call finds the scratch dirty
from the first).  This file is collected last so that a run stopping at the
first failure has run every other test already; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


def _reference_rows(scene, cams, dev):
    """Row maps from the allocating path (mesh upload + sm_fuse_frames)."""
    from paper_2111_11103_gb300 import labelfuse as lf
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    V = torch.as_tensor(scene.vertices, device=dev)
    Fc = torch.as_tensor(scene.faces, device=dev)
    K = torch.as_tensor(cams.K, device=dev)
    T = torch.as_tensor(cams.cam_to_world.reshape(N, 16), device=dev)
    probs = torch.full((N, H, W, c), 1.0 / c, device=dev)
    idm = torch.empty((N, H, W), dtype=torch.int32, device=dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "sum", "pixel")
    try:
        lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W, idm)
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)
    return idm


@pytest.mark.parametrize("case", ["tiny", "medium"])
def test_noalloc_rows_match_fuse_frames(case):
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2111_11103_gb300 import labelfuse as lf
    dev = torch.device("cuda:0")
    if case == "tiny":
        scene, cams = sg.tiny_room(), sg.circle_poses()
    else:
        scene = sg.paper_room(target_faces=60_000)
        cams = sg.random_walk_poses(12, H=151, W=203, fx=183.0, fy=183.0, cx=101.0, cy=75.0)
    N, H, W = cams.K.shape[0], cams.H, cams.W
    ref = _reference_rows(scene, cams, dev)
    V = torch.as_tensor(scene.vertices, device=dev)
    Fc = torch.as_tensor(scene.faces, device=dev)
    K = torch.as_tensor(cams.K, device=dev)
    T = torch.as_tensor(cams.cam_to_world.reshape(N, 16), device=dev)
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_render_rows_noalloc(V, Fc, K, T, N, H, W, out)
        torch.cuda.synchronize(dev)
        assert torch.equal(out, ref), f"{(out != ref).sum().item()} pixels differ"
    assert (ref >= 0).float().mean().item() > 0.99


def test_noalloc_rejects_oversized_calls():
    from paper_2111_11103_gb300 import labelfuse as lf
    dev = torch.device("cuda:0")
    scene, cams = sg.tiny_room(), sg.circle_poses(n=1)
    V = torch.as_tensor(scene.vertices, device=dev)
    Fc = torch.as_tensor(scene.faces, device=dev)
    K = torch.as_tensor(cams.K, device=dev)
    T = torch.as_tensor(cams.cam_to_world.reshape(1, 16), device=dev)
    big = torch.empty(1, dtype=torch.int32, device=dev)
    with pytest.raises(lf.LabelFuseError):   # more pixels than the static z-buffer holds
        lf.sm_render_rows_noalloc(V, Fc, K, T, 1, 2048, 1024, big)
    with pytest.raises(lf.LabelFuseError):   # more frames than the static camera slots
        lf.sm_render_rows_noalloc(V, Fc, K, T, lf.SM_NOALLOC_MAX_FRAMES + 1, 8, 8, big)
    with pytest.raises(lf.LabelFuseError):   # NULL output
        lf.sm_render_rows_noalloc(V, Fc, K, T, 1, 8, 8, None)
    # the rejected calls enqueued nothing; a valid call still matches afterwards
    ref = _reference_rows(scene, cams, dev)
    out = torch.empty_like(ref)
    lf.sm_render_rows_noalloc(V, Fc, K, T, 1, cams.H, cams.W, out)
    torch.cuda.synchronize(dev)
    assert torch.equal(out, ref)
