"""GPU parity of the learned confidence against its binary64 oracle:
features, the bfloat16 network's outputs, the training gradient and loss,
the agreement targets, fusion with the predicted per-pixel weights (every
rule), and a short training run lowering the loss."""
import numpy as np
import pytest
import torch

import scenegen as sg
from gpu_common import assert_acc_close, to_dev
from oracle import confidence as cf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2111_11103_gb300 import labelfuse as lf
    lf.lib()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def tiny(dev):
    scene, cams = sg.tiny_room(), sg.circle_poses()
    return scene, cams, sg.predictions(scene, cams, "tiny", device=dev)


@pytest.fixture(scope="module")
def medium(dev):
    scene = sg.paper_room(target_faces=60_000)
    cams = sg.random_walk_poses(12, H=151, W=203, fx=183.0, fy=183.0, cx=101.0, cy=75.0)
    return scene, cams, sg.predictions(scene, cams, "paper", device=dev)


def gpu_features(scene, cams, probs, dev):
    from paper_2111_11103_gb300 import labelfuse as lf
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "sum", "pixel")
    try:
        feat = torch.full((N, H, W, 5), -3.0, device=dev)
        rows = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_conf_features(m, probs, "f32", None, K, T, N, H, W, feat, rows)
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)
    return feat, rows


def _params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, cf.N_PARAMS).astype(np.float32)


@pytest.mark.parametrize("which", ["tiny", "medium"])
def test_features_match_oracle(ora, dev, tiny, medium, which):
    scene, cams, probs = tiny if which == "tiny" else medium
    feat, rows = gpu_features(scene, cams, probs, dev)
    feat, rows = feat.cpu().numpy(), rows.cpu().numpy()
    P = probs.cpu().numpy()
    for i in range(cams.K.shape[0]):
        X, face = cf.features(ora, scene.vertices, scene.faces, cams.K[i], cams.cam_to_world[i], P[i], cams.H, cams.W)
        assert np.array_equal(rows[i].ravel(), face)  # face mode: row = triangle
        np.testing.assert_allclose(feat[i].reshape(-1, 5), X, rtol=0, atol=3e-6)


def test_forward_and_gradient_match_oracle(dev, medium):
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    feat, rows = gpu_features(scene, cams, probs, dev)
    X = feat.reshape(-1, 5)[rows.reshape(-1) >= 0][:5000].contiguous()
    n = X.shape[0]
    y = (torch.arange(n, device=dev) % 3 == 0).float()
    params = torch.as_tensor(_params(3), device=dev)
    w = torch.empty(n, device=dev)
    lf.sm_conf_forward(params, X, n, w)
    _, w_ora, _ = cf.forward(params.cpu().numpy(), X.cpu().numpy())
    np.testing.assert_allclose(w.cpu().numpy(), w_ora, rtol=1e-5, atol=2e-6)
    grad, loss = torch.empty(cf.N_PARAMS, device=dev), torch.empty(1, device=dev)
    p0 = params.clone()
    lf.sm_conf_train_step(params, X, y, n, 0.0, grad, loss)
    torch.cuda.synchronize()
    assert torch.equal(params, p0)  # lr = 0
    l_ora, g_ora = cf.loss_and_grad(p0.cpu().numpy(), X.cpu().numpy(), y.cpu().numpy())
    assert abs(float(loss) - l_ora) <= 1e-5 * abs(l_ora)
    np.testing.assert_allclose(grad.cpu().numpy(), g_ora, rtol=0, atol=1e-5 * np.abs(g_ora).max())
    grad2, loss2 = torch.empty_like(grad), torch.empty_like(loss)
    lf.sm_conf_train_step(params, X, y, n, 0.0, grad2, loss2)
    torch.cuda.synchronize()
    assert torch.equal(grad, grad2) and torch.equal(loss, loss2)  # fixed-point sums: reproducible bit for bit
    X_bad = X.clone()
    X_bad[7, 2] = float("nan")
    p_bad = p0.clone()
    lf.sm_conf_train_step(p_bad, X_bad, y, n, 0.5, grad2, loss2)
    torch.cuda.synchronize()
    assert torch.isnan(grad2).all() and torch.isnan(loss2).all()  # a non-finite partial sum poisons the step
    lf.sm_conf_train_step(params, X, y, n, 0.5, grad, loss)  # the update is params - lr * grad
    torch.cuda.synchronize()
    np.testing.assert_allclose(params.cpu().numpy(), p0.cpu().numpy() - 0.5 * grad.cpu().numpy(), rtol=0, atol=1e-7)


def test_indexed_step_equals_the_gathered_step(dev, medium):
    """A minibatch given by indices (repeats included) gives bit for bit the
    step on the gathered rows, whose gradient the test above checks against
    the oracle; the oracle's gradient of the gathered rows holds here too; an
    index outside the observations poisons the step instead of being read."""
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    feat, rows = gpu_features(scene, cams, probs, dev)
    X = feat.reshape(-1, 5)[rows.reshape(-1) >= 0][:20000].contiguous()
    n = X.shape[0]
    y = (torch.arange(n, device=dev) % 5 < 2).float()
    g = torch.Generator(device=dev).manual_seed(11)
    idx = torch.randint(0, n, (3000,), device=dev, generator=g)
    params = torch.as_tensor(_params(4), device=dev)
    p_a, p_b = params.clone(), params.clone()
    grad_a, loss_a = torch.empty(cf.N_PARAMS, device=dev), torch.empty(1, device=dev)
    grad_b, loss_b = torch.empty_like(grad_a), torch.empty_like(loss_a)
    Xg, yg = X[idx].contiguous(), y[idx].contiguous()
    lf.sm_conf_train_step(p_a, Xg, yg, idx.numel(), 0.25, grad_a, loss_a)
    lf.sm_conf_train_step_indexed(p_b, X, y, n, idx, idx.numel(), 0.25, grad_b, loss_b)
    torch.cuda.synchronize()
    assert torch.equal(grad_a, grad_b) and torch.equal(loss_a, loss_b) and torch.equal(p_a, p_b)
    l_ora, g_ora = cf.loss_and_grad(params.cpu().numpy(), Xg.cpu().numpy(), yg.cpu().numpy())
    assert abs(float(loss_b) - l_ora) <= 1e-5 * abs(l_ora)
    np.testing.assert_allclose(grad_b.cpu().numpy(), g_ora, rtol=0, atol=1e-5 * np.abs(g_ora).max())
    bad = idx.clone()
    bad[123] = n  # one past the end: not read, the step is poisoned
    lf.sm_conf_train_step_indexed(params.clone(), X, y, n, bad, bad.numel(), 0.25, grad_b, loss_b)
    torch.cuda.synchronize()
    assert torch.isnan(grad_b).all() and torch.isnan(loss_b).all()


@pytest.mark.parametrize("rule", ["sum", "logsum", "maxsum", "vote"])
def test_fusion_with_predicted_weights(ora, dev, tiny, rule):
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = tiny
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    feat, rows = gpu_features(scene, cams, probs, dev)
    params = torch.as_tensor(_params(4), device=dev)
    w = torch.empty((N, H, W), device=dev)
    lf.sm_conf_forward(params, feat, N * H * W, w)
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, rule, "pixel")
    try:
        lf.sm_fuse_frames_weighted(m, probs, "f32", None, K, T, N, H, W, w)
        acc = torch.empty((len(scene.faces), c), device=dev)
        cnt = torch.empty(len(scene.faces), dtype=torch.int32, device=dev)
        lf.sm_read_state(m, acc, cnt)
        lf.sm_check(m)
        with pytest.raises(lf.LabelFuseError):
            lf.sm_fuse_frames_weighted(m, probs, "f32", None, K, T, N, H, W, None)
    finally:
        lf.sm_mesh_free(m)
    A, cnt_o = ora.accumulate(rule, rows.cpu().numpy().ravel(), probs.cpu().numpy().reshape(-1, c), len(scene.faces),
                              weights=w.cpu().numpy().ravel().astype(np.float64))
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), cnt_o)
    assert_acc_close(acc.cpu().numpy(), A)


def test_targets_and_training_lower_the_loss(ora, dev, medium):
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    feat, rows = gpu_features(scene, cams, probs, dev)
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "logsum", "pixel")
    try:
        lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W)
        labels = torch.empty(len(scene.faces), dtype=torch.int32, device=dev)
        lf.sm_normalise(m, None, labels)
        y = torch.empty((N, H, W), device=dev)
        lf.sm_conf_targets(m, probs, "f32", None, rows, N * H * W, y)
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)
    y_ora = cf.targets(probs.cpu().numpy().reshape(-1, c), rows.cpu().numpy().ravel(), labels.cpu().numpy())
    assert np.array_equal(y.cpu().numpy().ravel(), y_ora)
    sel = rows.reshape(-1) >= 0
    X, Y = feat.reshape(-1, 5)[sel].contiguous(), y.reshape(-1)[sel].contiguous()
    params = torch.as_tensor(_params(5, 0.2), device=dev)
    grad, loss = torch.empty(cf.N_PARAMS, device=dev), torch.empty(1, device=dev)
    losses = []
    for _ in range(150):
        lf.sm_conf_train_step(params, X, Y, X.shape[0], 1.0, grad, loss)
        losses.append(float(loss))
    assert losses[-1] < 0.9 * losses[0]
    assert np.isfinite(losses).all()


def test_fused_inference_matches_oracle(ora, dev, medium):
    """sm_conf_weights (features and network in one pass, hidden layer on the
    tensor cores): row maps bit for bit; weights against the oracle's network
    with the first layer's activations rounded to bfloat16 (as the tensor
    cores take them), and against the float32-activation forward pass
    (sm_conf_forward) within 1.6e-2.  Against the oracle the bound is per
    observation: an activation computed in float32 on the GPU and in binary64
    in the oracle may round to neighbouring bfloat16 values (at most 2^-6 |h1|
    apart), which moves o, and so w = max(o, 1/16), by at most
    sum_i 2^-6 |h1_i| (|W2|^T |w3|)_i; almost every observation matches far
    closer."""
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    params = torch.as_tensor(_params(6, 0.3), device=dev)
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    m = lf.sm_mesh_upload(V, Fc, None, c, "sum", "pixel")
    try:
        w = torch.full((N, H, W), -1.0, device=dev)
        rows = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_conf_weights(m, probs, "f32", None, K, T, N, H, W, params, w, rows)
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)
    feat, rows_f = gpu_features(scene, cams, probs, dev)
    assert torch.equal(rows, rows_f)
    w_fp32 = torch.empty((N, H, W), device=dev)
    lf.sm_conf_forward(params, feat, N * H * W, w_fp32)
    w, rows, w_fp32 = w.cpu().numpy(), rows.cpu().numpy(), w_fp32.cpu().numpy()
    assert np.all(w[rows < 0] == 0.0)
    fg = rows >= 0
    np.testing.assert_allclose(w[fg], w_fp32[fg], rtol=0, atol=1.6e-2)
    P = probs.cpu().numpy()
    for i in range(N):
        X, face = cf.features(ora, scene.vertices, scene.faces, cams.K[i], cams.cam_to_world[i], P[i], H, W)
        assert np.array_equal(rows[i].ravel(), face)
        _, w_ora, (_, _, h1, _, _) = cf.forward(params.cpu().numpy(), X, act_bf16=True)
        W1, b1, W2, b2, w3, b3 = cf.unpack(cf.bf16_round(params.cpu().numpy()))
        bound = (2.0 ** -6 * np.abs(h1)) @ (np.abs(W2).T @ np.abs(w3)) + 4e-5
        sel = face >= 0
        err = np.abs(w[i].ravel()[sel] - w_ora[sel])
        assert np.all(err <= bound[sel]), (err.max(), bound[sel][np.argmax(err - bound[sel])])
        assert err.mean() <= 8e-6, err.mean()


@pytest.mark.parametrize("mode,rule", [("face", "logsum"), ("face", "sum"), ("texel", "logsum"), ("texel", "maxsum")])
def test_one_pass_confident_fusion(ora, dev, medium, mode, rule):
    """sm_fuse_frames_confident (raster, weights, weighted scatter per batch)
    against the two passes it replaces (sm_conf_weights, then
    sm_fuse_frames_weighted): the same weights and row maps bit for bit, the
    same counts, accumulators within float32 summation order; and against the
    oracle: its row maps (texel rows in texel mode, which sm_conf_weights now
    also writes) and its weighted accumulation of the GPU's weights.  Batches
    of 8 frames, so the 12 frames take two launches, the second one short."""
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, probs = medium
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    tres = None
    if mode == "texel":
        tres = np.random.default_rng(11).integers(1, 4, len(scene.faces)).astype(np.int32)
    params = torch.as_tensor(_params(8, 0.3), device=dev)
    V, Fc, K, T, tr = to_dev(scene, cams, tres, dev)
    m = lf.sm_mesh_upload(V, Fc, tr, c, rule, "pixel")
    n_x = lf.sm_num_rows(m)
    try:
        lf.sm_set_launch_frames(m, H, W, 8)
        w_a = torch.full((N, H, W), -1.0, device=dev)
        rows_a = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        idm_a = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_conf_weights(m, probs, "f32", None, K, T, N, H, W, params, w_a, rows_a)
        lf.sm_fuse_frames_weighted(m, probs, "f32", None, K, T, N, H, W, w_a, idm_a)
        acc_a = torch.empty((n_x, c), device=dev)
        cnt_a = torch.empty(n_x, dtype=torch.int32, device=dev)
        lf.sm_read_state(m, acc_a, cnt_a)
        lf.sm_reset(m)
        w_b = torch.full((N, H, W), -1.0, device=dev)
        idm_b = torch.full((N, H, W), -7, dtype=torch.int32, device=dev)
        lf.sm_fuse_frames_confident(m, probs, "f32", None, K, T, N, H, W, params, w_b, idm_b)
        acc_b = torch.empty((n_x, c), device=dev)
        cnt_b = torch.empty(n_x, dtype=torch.int32, device=dev)
        lf.sm_read_state(m, acc_b, cnt_b)
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)
    assert torch.equal(w_a, w_b)
    assert torch.equal(rows_a, idm_a) and torch.equal(idm_a, idm_b)
    assert torch.equal(cnt_a, cnt_b)
    torch.testing.assert_close(acc_b, acc_a, rtol=1e-5, atol=1e-6)
    mesh = ora.Mesh(scene.vertices, scene.faces, tres)
    rows_o = ora.render_sequence(mesh, cams.K, cams.cam_to_world, H, W)
    idm = idm_b.cpu().numpy()
    assert np.array_equal(idm, rows_o)
    w = w_b.cpu().numpy()
    assert np.all(w[idm < 0] == 0.0) and np.all(w[idm >= 0] >= 0.0625)
    A, cnt = ora.accumulate(rule, rows_o, probs.cpu().numpy(), mesh.n_x, weights=w.astype(np.float64))
    assert np.array_equal(cnt_b.cpu().numpy().astype(np.int64), cnt)
    assert_acc_close(acc_b.cpu().numpy(), A)


def test_learned_confidence_gains_over_plain_fusion(dev):
    """The network's gain: predictions whose errors follow the view (the
    "structured" recipe: confidently wrong more often at grazing angles, far
    away and near the image border).  The network is trained on agreement
    with the plain fused labels; the render-back pixel accuracy against the
    synthetic ground truth of the weighted fusion (weights max(o, 1/16), the
    floored log-odds of agreement) must beat plain fusion by half a point,
    for each of three training seeds (initial parameters and minibatches)."""
    from paper_2111_11103_gb300 import confidence as conf
    from paper_2111_11103_gb300 import labelfuse as lf
    scene = sg.paper_room(target_faces=60_000)
    cams = sg.random_walk_poses(24, H=151, W=203, fx=183.0, fy=183.0, cx=101.0, cy=75.0)
    N, H, W, c = cams.K.shape[0], cams.H, cams.W, scene.n_classes
    probs = sg.predictions(scene, cams, "structured", device=dev)
    gt = torch.stack([sg.ray_cast_classes(scene, cams.K[i], cams.cam_to_world[i], H, W, device=dev)
                      for i in range(N)])
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    seen = gt >= 0
    idm = torch.empty((N, H, W), dtype=torch.int32, device=dev)
    img = torch.empty((N, H, W), dtype=torch.uint8, device=dev)
    acc = {}
    m = lf.sm_mesh_upload(V, Fc, None, c, "logsum", "pixel")
    try:
        lf.sm_fuse_frames(m, probs, "f32", None, K, T, N, H, W, idm)
        lf.sm_normalise(m)
        lf.sm_render_idmap(m, idm, N * H * W, img)
        acc["plain"] = float((img.long()[seen] == gt[seen]).float().mean())
        for seed in (0, 1, 2):
            params, losses = conf.train(m, probs, K, T, H, W, steps=2000, lr=1.0, batch=200_000, seed=seed)
            assert losses[-1] < losses[0]
            lf.sm_reset(m)
            conf.fuse_with_confidence(m, params, probs, K, T, H, W, idmap_out=idm)
            lf.sm_normalise(m)
            lf.sm_render_idmap(m, idm, N * H * W, img)
            acc[seed] = float((img.long()[seen] == gt[seen]).float().mean())
        lf.sm_check(m)
    finally:
        lf.sm_mesh_free(m)
    raw = float((probs.argmax(-1)[seen] == gt[seen]).float().mean())
    print(f"pixel accuracy: raw {raw:.4f}, plain fusion {acc['plain']:.4f}, weighted "
          + ", ".join(f"{acc[s]:.4f} (seed {s})" for s in (0, 1, 2)))
    for seed in (0, 1, 2):
        assert acc[seed] >= acc["plain"] + 0.005, (seed, acc)
