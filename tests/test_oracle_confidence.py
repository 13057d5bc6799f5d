"""Pins for the confidence oracle: gradients against central finite
differences, closed-form forward passes, bfloat16 rounding against torch's
own conversion, and features with closed forms (a fronto-parallel wall,
uniform / one-hot predictions, hand-worked border distances)."""
import numpy as np
import torch

from oracle import confidence as cf


def _random_params(rng, scale=0.4):
    return cf.bf16_round(rng.normal(0, scale, cf.N_PARAMS).astype(np.float32))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    params = _random_params(rng)
    X = rng.uniform(0, 1, (64, cf.N_FEAT))
    y = (rng.uniform(size=64) < 0.6).astype(np.float64)
    _, g = cf.loss_and_grad(params, X, y, rounding=False)
    eps = 1e-6
    idx = rng.choice(cf.N_PARAMS, 120, replace=False)
    for i in idx:
        d = np.zeros(cf.N_PARAMS)
        d[i] = eps
        lp, _ = cf.loss_and_grad(params + d, X, y, rounding=False)
        lm, _ = cf.loss_and_grad(params - d, X, y, rounding=False)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_forward_closed_forms():
    p = np.zeros(cf.N_PARAMS)
    p[-1] = 0.75  # b3: o = 0.75 for every input, the weight is the log-odds itself
    o, w, _ = cf.forward(p, np.ones((3, cf.N_FEAT)))
    assert np.array_equal(o, [0.75] * 3) and np.array_equal(w, [0.75] * 3)
    p[-1] = -0.75  # below even odds: the floor of 1/16
    o, w, _ = cf.forward(p, np.ones((3, cf.N_FEAT)))
    assert np.array_equal(o, [-0.75] * 3) and np.array_equal(w, [0.0625] * 3)
    # the loss at o = b3 is the BCE of the constant probability sigmoid(b3)
    y = np.array([1.0, 0.0, 1.0])
    l, g = cf.loss_and_grad(p, np.ones((3, cf.N_FEAT)), y)
    q = 1 / (1 + np.exp(0.75))
    assert abs(l - np.mean(-(y * np.log(q) + (1 - y) * np.log(1 - q)))) <= 1e-15
    assert abs(g[-1] - np.mean(q - y)) <= 1e-15  # d loss / d b3
    # one path through: o = relu(relu(x0)) = x0 for x0 >= 0, 0 for x0 < 0; w = max(o, 1/16)
    W1, b1, W2, b2, w3, b3 = cf.unpack(np.zeros(cf.N_PARAMS))
    q = np.zeros(cf.N_PARAMS)
    q[0] = 1.0                                   # W1[0, 0]
    q[cf.HID * cf.N_FEAT + cf.HID] = 1.0         # W2[0, 0]
    q[cf.N_PARAMS - 1 - cf.HID] = 1.0            # w3[0]
    X = np.array([[0.5, 9, 9, 9, 9], [-2.0, 1, 1, 1, 1]])
    o, w, _ = cf.forward(q, X)
    assert np.array_equal(o, [0.5, 0.0]) and np.array_equal(w, [0.5, 0.0625])


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = (rng.normal(0, 1, 20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cf.bf16_round(x), ref)
    # exact ties (low half 0x8000) go to the even neighbour; 0x7FFF / 0x8001 round down / up
    hi = rng.integers(0x0080, 0x7F00, 4000, dtype=np.uint32) << 16
    for low in (0x8000, 0x7FFF, 0x8001):
        t = (hi | np.uint32(low)).view(np.float32)
        ref = torch.from_numpy(t.copy()).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(cf.bf16_round(t), ref)


def test_features_fronto_parallel_wall(ora):
    """Wall at z = 2 facing the camera (identity pose): depth feature 2/4,
    |cos| = 1 / |((x-cx)/fx, (y-cy)/fy, 1)|, border distance by hand."""
    V = np.array([[-1, -0.75, 2], [1, -0.75, 2], [1, 0.75, 2], [-1, 0.75, 2]], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 2, 3]])
    K = np.array([10.0, 10.0, 8.25, 6.25])
    H, W, c = 14, 18, 4
    probs = np.full((H, W, c), 0.25, dtype=np.float32)   # uniform: entropy 1, margin 0
    probs[3, 4] = [1, 0, 0, 0]                           # one-hot: entropy 0, margin 1
    X, face = cf.features(ora, V, F, K, np.eye(4), probs, H, W)
    X = X.reshape(H, W, 5)
    cov = face.reshape(H, W) >= 0
    assert np.all(X[cov, 1] == 0.5)
    ys, xs = np.mgrid[0:H, 0:W]
    cos = 1 / np.sqrt(((xs - 8.25) / 10) ** 2 + ((ys - 6.25) / 10) ** 2 + 1)
    np.testing.assert_allclose(X[cov, 0], cos[cov], rtol=1e-14)
    assert X[3, 4, 2] == 0.0 and X[3, 4, 3] == 1.0
    np.testing.assert_allclose(X[5, 5, 2], 1.0, rtol=1e-12)
    assert X[5, 5, 3] == 0.0
    assert X[3, 4, 4] == 3 / 7 and X[9, 13, 4] == 4 / 7  # min(4,3,13,10) = 3; min(13,9,4,4) = 4; / (14/2)
    assert np.all(X[~cov] == 0)
    # the view-angle feature does not depend on the winding (the sign of the normal)
    X2, face2 = cf.features(ora, V, F[:, [0, 2, 1]], K, np.eye(4), probs, H, W)
    assert np.array_equal(face2, face) and np.array_equal(X2.reshape(H, W, 5), X)


def test_targets_by_hand():
    probs = np.array([[0.1, 0.7, 0.2], [0.5, 0.5, 0.0], [0.2, 0.3, 0.5], [0.6, 0.3, 0.1]])
    rows = np.array([0, 1, 1, -1])
    labels = np.array([1, 0])
    assert list(cf.targets(probs, rows, labels)) == [1.0, 1.0, 0.0, 0.0]


def test_forward_with_bfloat16_activations():
    """act_bf16 rounds exactly the first layer's activations: with
    activations that are already bfloat16 values it changes nothing, and
    otherwise it moves w by no more than the rounding can (2^-9 relative per
    activation through the two later layers)."""
    rng = np.random.default_rng(11)
    params = rng.normal(0, 0.3, cf.N_PARAMS)
    X = rng.uniform(0, 1, (400, cf.N_FEAT))
    o, w, (_, z1, h1, z2, h2) = cf.forward(params, X)
    o_b, w_b, (_, _, h1_b, _, _) = cf.forward(params, X, act_bf16=True)
    assert np.array_equal(h1_b, cf.bf16_round(h1))
    W1, b1, W2, b2, w3, b3 = cf.unpack(cf.bf16_round(params))
    bound = (np.abs(h1) * 2.0 ** -8) @ np.abs(W2).T @ np.abs(w3)
    assert np.all(np.abs(o_b - o) <= bound + 1e-12)
    # a first layer whose activations are exact bfloat16 values: identical
    p2 = params.copy()
    p2[:cf.HID * cf.N_FEAT] = 0.0
    p2[cf.HID * cf.N_FEAT:cf.HID * cf.N_FEAT + cf.HID] = cf.bf16_round(rng.normal(0, 1, cf.HID))
    assert np.array_equal(cf.forward(p2, X)[0], cf.forward(p2, X, act_bf16=True)[0])
