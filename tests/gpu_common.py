"""Helpers for the GPU parity tests: run the CUDA library through its C ABI and
compare with the oracle under the acceptance rules:

* row maps and render-back of identical labels: bit for bit;
* accumulators: |A_gpu - A_ora| <= 1e-5 * max(|A_ora|, 1e-30) per class;
* labels: identical except rows whose oracle top-2 margin is below 1e-4
  (normalised distribution for sum/maxsum/vote; (L1 - L2) / max(1, |L1|) on
  the log accumulator for logsum);
* observation counts: exact.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

REL_TOL = 1e-5
MARGIN = 1e-4


@dataclasses.dataclass
class GpuResult:
    idmaps: np.ndarray
    acc: np.ndarray
    cnt: np.ndarray
    dist: np.ndarray
    labels: np.ndarray
    images: np.ndarray
    images_reraster: np.ndarray | None
    n_x: int


def to_dev(scene, cams, texel_res=None, dev="cuda"):
    N = cams.K.shape[0]
    V = torch.as_tensor(np.ascontiguousarray(scene.vertices), device=dev)
    Fc = torch.as_tensor(np.ascontiguousarray(scene.faces), device=dev)
    K = torch.as_tensor(np.ascontiguousarray(cams.K), device=dev)
    T = torch.as_tensor(np.ascontiguousarray(cams.cam_to_world.reshape(N, 16)), device=dev)
    tr = None if texel_res is None else torch.as_tensor(np.ascontiguousarray(texel_res, dtype=np.int32), device=dev)
    return V, Fc, K, T, tr


def run_gpu(scene, cams, probs, rule, weight, texel_res=None, dtype="f32", scale=None, reraster=True,
            n_classes=None, alpha=None, queue_shape=None, buffers="torch"):
    """Fuses, normalises and renders through the C ABI.  queue_shape: None
    (the library's choice), 0 (the two-stream path) or (frames per batch,
    lookahead, raster rounds, scatter tiles) of the work-queue path.
    buffers: "torch" or "compressible" (row maps and label images in the
    library's sm_device_alloc memory)."""
    from paper_2111_11103_gb300 import labelfuse as lf
    dev = probs.device
    N, H, W = cams.K.shape[0], cams.H, cams.W
    c = n_classes or scene.n_classes
    V, Fc, K, T, tr = to_dev(scene, cams, texel_res, dev)
    m = lf.sm_mesh_upload(V, Fc, tr, c, rule, weight)
    try:
        if alpha is not None:
            lf.sm_set_weight_mix(m, alpha)
        if queue_shape is not None:
            lf.sm_set_queue_shape(m, H, W, *((0,) if queue_shape == 0 else tuple(queue_shape)))
        n_x = lf.sm_num_rows(m)
        if buffers == "compressible":
            idm = lf.device_empty((N, H, W), torch.int32, dev).fill_(-7)
        else:
            idm = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_fuse_frames(m, probs, dtype, scale, K, T, N, H, W, idm)
        acc = torch.empty((max(n_x, 1), c), dtype=torch.float32, device=dev)
        cnt = torch.empty(max(n_x, 1), dtype=torch.int32, device=dev)
        lf.sm_read_state(m, acc, cnt)
        dist = torch.empty((max(n_x, 1), c), dtype=torch.float32, device=dev)
        labels = torch.empty(max(n_x, 1), dtype=torch.int32, device=dev)
        lf.sm_normalise(m, dist, labels)
        if buffers == "compressible":
            img = lf.device_empty((N, H, W), torch.uint8, dev)
        else:
            img = torch.empty((N, H, W), dtype=torch.uint8, device=dev)
        lf.sm_render_idmap(m, idm, N * H * W, img)
        img2 = None
        if reraster:
            img2 = torch.empty((N, H, W), dtype=torch.uint8, device=dev)
            idm2 = torch.empty((N, H, W), dtype=torch.int32, device=dev)
            lf.sm_render_labels(m, K, T, N, H, W, img2, idm2)
        lf.sm_check(m)
        if reraster:
            assert torch.equal(idm2, idm), "re-rendered row maps differ from the fused ones"
    finally:
        lf.sm_mesh_free(m)
    return GpuResult(idm.cpu().numpy(), acc.cpu().numpy()[:n_x], cnt.cpu().numpy()[:n_x].astype(np.int64),
                     dist.cpu().numpy()[:n_x], labels.cpu().numpy()[:n_x], img.cpu().numpy(),
                     None if img2 is None else img2.cpu().numpy(), n_x)


def assert_acc_close(acc_gpu, A_ora, rows=None):
    a = acc_gpu.astype(np.float64)
    A = A_ora if rows is None else A_ora[rows]
    a = a if rows is None else a[rows]
    err = np.abs(a - A)
    bound = REL_TOL * np.maximum(np.abs(A), 1e-30)
    bad = err > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{bad.sum()} accumulator entries outside 1e-5 relative; first at {tuple(i)}: "
                             f"gpu {a[tuple(i)]!r} oracle {A[tuple(i)]!r}")


def top2_margin(rule, A, dist):
    """Oracle's top-2 margin per row (see module docstring)."""
    if A.shape[1] < 2:
        return np.full(A.shape[0], np.inf)
    if rule == "logsum":
        s = np.sort(A, axis=1)
        return (s[:, -1] - s[:, -2]) / np.maximum(1.0, np.abs(s[:, -1]))
    s = np.sort(dist, axis=1)
    return s[:, -1] - s[:, -2]


def assert_labels_match(rule, labels_gpu, A, cnt, dist_ora, labels_ora):
    margin = top2_margin(rule, A, dist_ora)
    diff = (labels_gpu != labels_ora)
    unseen = cnt == 0
    assert np.all(labels_gpu[unseen] == -1)
    allowed = margin < MARGIN
    bad = diff & ~allowed
    assert not bad.any(), f"{bad.sum()} labels differ on rows with margin >= {MARGIN}"
    return int(diff.sum())


def check_against_oracle(ora, scene, cams, probs_np, res: GpuResult, rule, weight, texel_res=None,
                         nthreads=4, alpha=1.0):
    """Full comparison on a case small enough for the oracle."""
    mesh = ora.Mesh(scene.vertices, scene.faces, texel_res=texel_res)
    assert mesh.n_x == res.n_x
    A, cnt, idm = ora.fuse_sequence(mesh, cams.K, cams.cam_to_world, probs_np, rule, weight, nthreads=nthreads,
                                    want_idmaps=True, alpha=alpha)
    assert np.array_equal(res.idmaps, idm), f"{(res.idmaps != idm).sum()} row-map pixels differ"
    assert np.array_equal(res.cnt, cnt), "observation counts differ"
    assert_acc_close(res.acc, A)
    dist, lab = ora.normalise(rule, A, cnt)
    ndiff = assert_labels_match(rule, res.labels, A, cnt, dist, lab)
    # render-back of the GPU's labels through the oracle's row maps: bit for bit
    assert np.array_equal(ora.render_labels(idm, res.labels), res.images)
    if res.images_reraster is not None:
        assert np.array_equal(res.images_reraster, res.images)
    check_distributions(rule, res, cnt, dist)
    return ndiff


def check_distributions(rule, res: GpuResult, cnt, dist_ora=None):
    """The GPU's normalisation is the normalisation of its own accumulators
    (recomputed here in binary64); for the additive rules it also matches the
    oracle's distributions.  For logsum the distribution exp(L - max L) / sum
    amplifies the accumulators' rounding by |L|, so only the accumulators are
    held to the oracle."""
    seen = cnt > 0
    assert np.all(res.dist[~seen] == 0)
    if not seen.any():
        return
    a = res.acc[seen].astype(np.float64)
    if rule == "logsum":
        e = np.exp(a - a.max(1, keepdims=True))
        ref = e / e.sum(1, keepdims=True)
    else:
        ref = a / a.sum(1, keepdims=True)
    np.testing.assert_allclose(res.dist[seen], ref, atol=2e-6)
    np.testing.assert_allclose(res.dist[seen].sum(1), 1.0, atol=1e-5)
    if dist_ora is not None and rule != "logsum":
        np.testing.assert_allclose(res.dist[seen], dist_ora[seen], atol=2e-5)
