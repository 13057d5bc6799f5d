"""Full-size parity on the paper-shaped workload (the benchmark's workload and
launch configuration): 6 x 5 x 3 m room with boxes (~500k triangles), 1,000
frames of 640 x 480, c = 40, log-sum fusion with w^(P).

The oracle renders all 1,000 frames itself (threaded over frames) and
checks: every row map bit for bit, every row's observation count exactly,
the accumulators and labels of a sample of rows (the oracle accumulates
only the pixels that land on sampled rows, gathered from the same input
tensor), and every label image of the render-back bit for bit."""
import os

import numpy as np
import pytest
import torch

import scenegen as sg
from gpu_common import REL_TOL, assert_labels_match

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_paper_workload_full_size(ora):
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2111_11103_gb300 import labelfuse as lf
    dev = torch.device("cuda:0")
    scene = sg.paper_room()
    cams = sg.random_walk_poses(1000)
    N, H, W, c = 1000, cams.H, cams.W, scene.n_classes
    probs = torch.empty((N, H, W, c), dtype=torch.float32, device=dev)
    for a in range(0, N, 25):
        sg.predictions(scene, cams, "paper", frames=range(a, min(N, a + 25)), device=dev, out=probs[a:a + 25])
    V = torch.as_tensor(scene.vertices, device=dev)
    Fc = torch.as_tensor(scene.faces, device=dev)
    K = torch.as_tensor(cams.K, device=dev)
    T = torch.as_tensor(cams.cam_to_world.reshape(N, 16), device=dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "logsum", "pixel")
    try:
        n_x = lf.sm_num_rows(m)
        idm = torch.empty((N, H, W), dtype=torch.int32, device=dev)
        lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W, idm)
        acc = torch.empty((n_x, c), device=dev)
        cnt = torch.empty(n_x, dtype=torch.int32, device=dev)
        lf.sm_read_state(m, acc, cnt)
        labels = torch.empty(n_x, dtype=torch.int32, device=dev)
        lf.sm_normalise(m, None, labels)
        img = torch.empty((N, H, W), dtype=torch.uint8, device=dev)
        lf.sm_render_idmap(m, idm, N * H * W, img)
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)

    mesh = ora.Mesh(scene.vertices, scene.faces)
    idm_o = ora.render_sequence(mesh, cams.K, cams.cam_to_world, H, W, nthreads=os.cpu_count() or 1)
    idm_g = idm.cpu().numpy()
    assert np.array_equal(idm_g, idm_o), f"{(idm_g != idm_o).sum()} row-map pixels differ"

    cnt_o = np.bincount(idm_o[idm_o >= 0].ravel(), minlength=n_x)
    cnt_g = cnt.cpu().numpy().astype(np.int64)
    assert np.array_equal(cnt_g, cnt_o)
    assert cnt_o.sum() == (idm_o >= 0).sum()

    # accumulators and labels of a sample of observed rows
    rng = np.random.default_rng(11)
    seen = np.flatnonzero(cnt_o > 0)
    sample = rng.choice(seen, size=min(400, seen.size), replace=False)
    lut = np.zeros(n_x, dtype=bool)
    lut[sample] = True
    flat = idm_o.ravel()
    pix = np.flatnonzero((flat >= 0) & lut[np.maximum(flat, 0)])
    p_sel = probs.view(-1, c)[torch.as_tensor(pix, device=dev)].cpu().numpy()
    A, cnt_s = ora.accumulate("logsum", flat[pix], p_sel, n_x)
    assert np.array_equal(cnt_s[sample], cnt_o[sample])
    a_g = acc.cpu().numpy().astype(np.float64)
    err = np.abs(a_g[sample] - A[sample])
    bound = REL_TOL * np.maximum(np.abs(A[sample]), 1e-30)
    assert np.all(err <= bound), f"max relative error {np.max(err / np.maximum(np.abs(A[sample]), 1e-30)):.3g}"
    dist_o, lab_o = ora.normalise("logsum", A[sample], cnt_o[sample])
    lab_g = labels.cpu().numpy()
    assert_labels_match("logsum", lab_g[sample], A[sample], cnt_o[sample], dist_o, lab_o)
    assert np.all(lab_g[cnt_o == 0] == -1)

    # render-back of the GPU's labels through the oracle's row maps
    del probs
    torch.cuda.empty_cache()
    assert np.array_equal(ora.render_labels(idm_o, lab_g), img.cpu().numpy())


@pytest.mark.parametrize("kind", ["f32", "fp8_e4m3"])
def test_high_resolution_frames(ora, kind):
    """The high-resolution configuration's frames (1296 x 968, fx = fy = 1170,
    the full paper-shaped mesh): 6 frames against the oracle, FP32 and the
    FP8 storage form (the oracle fed the dequantised values)."""
    from gpu_common import check_against_oracle, run_gpu
    dev = torch.device("cuda:0")
    scene = sg.paper_room()
    cams = sg.random_walk_poses(6, H=968, W=1296, fx=1170.0, fy=1170.0, cx=647.5, cy=483.5)
    probs = sg.predictions(scene, cams, "paper", device=dev)
    if kind == "f32":
        res = run_gpu(scene, cams, probs, "logsum", "pixel", reraster=True)
        check_against_oracle(ora, scene, cams, probs.cpu().numpy(), res, "logsum", "pixel", nthreads=8)
    else:
        scale = probs.amax(-1) / 448.0
        q = (probs / scale[..., None]).to(torch.float8_e4m3fn).contiguous()
        deq = (q.float() * scale[..., None]).cpu().numpy()
        res = run_gpu(scene, cams, q, "sum", "pixel", dtype=kind, scale=scale.contiguous(), reraster=False)
        check_against_oracle(ora, scene, cams, deq, res, "sum", "pixel", nthreads=8)
    assert (res.idmaps >= 0).mean() > 0.99
