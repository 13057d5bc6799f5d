"""The allocation-free entry point sm_render_rows_noalloc.

It serves callers that cannot allocate device memory (a plugin whose host
application owns all device memory through its own pool, or a latency-bound
loop that must not call cudaMalloc, which can block and synchronise the
device).  It renders row maps with the library's static scratch instead.  Its
output must equal the row maps of the allocating entry point sm_fuse_frames
bit for bit, and the oracle's row maps, on two calls in a row (the second
call finds the scratch dirty from the first).  This file is collected last so
that a run stopping at the first failure has run every other test already; it
also passes on its own.
"""
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


def _inputs(scene, cams, dev):
    N = cams.K.shape[0]
    return (torch.as_tensor(scene.vertices, device=dev), torch.as_tensor(scene.faces, device=dev),
            torch.as_tensor(cams.K, device=dev), torch.as_tensor(cams.cam_to_world.reshape(N, 16), device=dev))


@pytest.mark.parametrize("case", ["tiny", "medium"])
def test_noalloc_rows_match_fuse_frames_and_oracle(ora, case):
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
    expect = ora.render_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world, H, W, nthreads=8)
    V, Fc, K, T = _inputs(scene, cams, dev)
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_render_rows_noalloc(V, Fc, K, T, N, H, W, out)
        torch.cuda.synchronize(dev)
        assert torch.equal(out, ref), f"{(out != ref).sum().item()} pixels differ from sm_fuse_frames"
        got = out.cpu().numpy()
        assert np.array_equal(got, expect), f"{(got != expect).sum()} pixels differ from the oracle"
    assert (ref >= 0).float().mean().item() > 0.99


def test_noalloc_limits_are_checked_by_the_library():
    """The library itself (not the binding's size checks) rejects calls beyond
    the static scratch, an output that is not device memory and inputs that are
    not memory of the output's device, before anything is enqueued.  Raw
    addresses bypass the binding's checks; the buffers behind them are real
    but small, which is safe because the library refuses before touching them."""
    from paper_2111_11103_gb300 import labelfuse as lf
    dev = torch.device("cuda:0")
    scene, cams = sg.tiny_room(), sg.circle_poses(n=1)
    V, Fc, K, T = _inputs(scene, cams, dev)
    small = torch.empty(64, dtype=torch.int32, device=dev)
    raw = small.data_ptr()
    h, w = 1024, lf.SM_NOALLOC_MAX_PIXELS // 1024 + 1    # one pixel row past the z-buffer
    host_out = torch.empty(64, dtype=torch.int32)
    host_K = torch.as_tensor(cams.K).contiguous()
    cases = {
        "pixels": (V, Fc, K, T, 1, h, w, raw),
        "frames": (V, Fc, K.data_ptr(), T.data_ptr(), lf.SM_NOALLOC_MAX_FRAMES + 1, 8, 8, raw),
        "host output": (V, Fc, K, T, 1, 8, 8, host_out.data_ptr()),
        "host cameras": (V, Fc, host_K.data_ptr(), T, 1, 8, 8, raw),
    }
    for name, args in cases.items():
        with pytest.raises(lf.LabelFuseError) as ei:
            lf.sm_render_rows_noalloc(*args)
        assert ei.value.status == lf.SM_ERR_INVALID_ARG, name
    torch.cuda.synchronize(dev)
    # the rejected calls enqueued nothing; a valid call still matches afterwards
    ref = _reference_rows(scene, cams, dev)
    out = torch.empty_like(ref)
    lf.sm_render_rows_noalloc(V, Fc, K, T, 1, cams.H, cams.W, out)
    torch.cuda.synchronize(dev)
    assert torch.equal(out, ref)


def test_noalloc_at_the_size_limit(ora):
    """Frames of exactly SM_NOALLOC_MAX_PIXELS pixels (1536 x 1024) are
    accepted and match the oracle."""
    from paper_2111_11103_gb300 import labelfuse as lf
    dev = torch.device("cuda:0")
    scene = sg.paper_room(target_faces=20_000)
    H, W = 1024, lf.SM_NOALLOC_MAX_PIXELS // 1024
    cams = sg.random_walk_poses(2, H=H, W=W, fx=1170.0, fy=1170.0, cx=W / 2 - 0.5, cy=H / 2 - 0.5)
    V, Fc, K, T = _inputs(scene, cams, dev)
    out = torch.empty((2, H, W), dtype=torch.int32, device=dev)
    lf.sm_render_rows_noalloc(V, Fc, K, T, 2, H, W, out)
    torch.cuda.synchronize(dev)
    expect = ora.render_sequence(ora.Mesh(scene.vertices, scene.faces), cams.K, cams.cam_to_world, H, W, nthreads=8)
    assert np.array_equal(out.cpu().numpy(), expect)
