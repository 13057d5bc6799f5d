"""Oracle of the learned per-observation confidence (an extension of the
weighted fusion rules of Sec. 3.2.2: the weight of an observation is
predicted by a small network instead of being 1 or 1/|K_i ∩ K_x|).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): plain binary64
numpy, slow, written for checking by eye.

Features of the observation of pixel (x, y) of frame i, whose visible
triangle is t (all computed from the oracle's own raster):
  0  |cos| of the angle between t's normal and the viewing ray of the pixel
  1  depth z of the visible surface at the pixel (1 / interpolated 1/z) / 4 m
  2  entropy -sum_j p_j ln max(p_j, 2^-30) of the prediction, / ln c
  3  top-2 margin p_(1) - p_(2) of the prediction
  4  distance to the nearest image border, min(x, y, W-1-x, H-1-y) / (min(W, H) / 2)

Network 5 -> 32 -> 32 -> 1 with ReLU hidden layers and a linear output o,
read as the log-odds that the observation agrees with the fused label
(sigmoid(o) is that probability).  The fusion weight of the observation is
w = max(o, 1/16): the log-odds of agreement, clipped at a small floor so that
an observation no better than a coin toss has almost no say, while a row
whose every observation is predicted below even odds still takes the plain
vote of its observations instead of a tie.  For independent voters
choosing between two answers, weighing each vote by the log-odds of its
competence is the optimal decision rule (Nitzan and Paroush, Int. Econ. Rev.
23, 1982); the weighted log-sum of Eq. w-mul is such a vote.  Parameters are one flat
vector of 1,281 values in the order W1 (32 x 5, row = output), b1 (32),
W2 (32 x 32), b2 (32), w3 (32), b3 (1); the forward pass uses them rounded
to bfloat16 (round to nearest even).
Loss: mean binary cross-entropy softplus(o) - y o against a target y in {0, 1}
(the pixel's arg max agrees with the plain fusion's label of its row).
"""
from __future__ import annotations

import numpy as np

N_FEAT, HID = 5, 32
W_FLOOR = 0.0625  # 1/16: the least fusion weight of an observation
N_PARAMS = HID * N_FEAT + HID + HID * HID + HID + HID + 1
P_MIN = 2.0 ** -30


def bf16_round(x) -> np.ndarray:
    """float32 values rounded to the nearest bfloat16 (ties to even), as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == N_PARAMS
    i = 0
    out = []
    for shape in [(HID, N_FEAT), (HID,), (HID, HID), (HID,), (HID,), (1,)]:
        n = int(np.prod(shape))
        out.append(p[i:i + n].reshape(shape))
        i += n
    return out


def forward(params, X, rounding: bool = True, act_bf16: bool = False):
    """o and the fusion weight w = max(o, 1/16) for observations X (n x 5), with the parameters
    rounded to bfloat16 (rounding=False: as given, for finite differences);
    also returns the hidden activations for backward.  act_bf16: the first
    layer's activations are rounded to bfloat16 before the hidden layer, the
    precision of a hidden layer computed on bfloat16 tensor cores."""
    W1, b1, W2, b2, w3, b3 = unpack(bf16_round(params) if rounding else params)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    if act_bf16:
        h1 = bf16_round(h1)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ w3 + b3[0]
    w = np.maximum(o, W_FLOOR)
    return o, w, (X, z1, h1, z2, h2)


def loss_and_grad(params, X, y, rounding: bool = True):
    """Mean BCE over the n observations and its gradient with respect to the
    (bfloat16-rounded) parameters, flat, in the parameter order."""
    o, _, (X, z1, h1, z2, h2) = forward(params, X, rounding)
    q = 1.0 / (1.0 + np.exp(-o))  # sigmoid(o): the predicted probability of agreement
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    loss = np.mean(np.logaddexp(0.0, o) - y * o)
    W1, b1, W2, b2, w3, b3 = unpack(bf16_round(params) if rounding else params)
    d_o = (q - y) / n
    g_w3 = h2.T @ d_o
    g_b3 = np.array([d_o.sum()])
    d_z2 = np.outer(d_o, w3) * (z2 > 0)
    g_W2 = d_z2.T @ h1
    g_b2 = d_z2.sum(0)
    d_z1 = (d_z2 @ W2) * (z1 > 0)
    g_W1 = d_z1.T @ X
    g_b1 = d_z1.sum(0)
    return loss, np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, g_b3])


def features(ora, mesh_vertices, faces, K, T, probs, H: int, W: int):
    """Features (H*W x 5) and visible triangle (-1: background) of one frame;
    K = (fx, fy, cx, cy), T 4 x 4 camera-to-world, probs H x W x c."""
    V = np.asarray(mesh_vertices, dtype=np.float32).reshape(-1, 3)
    Fc = np.asarray(faces, dtype=np.int32).reshape(-1, 3)
    mesh = ora.Mesh(V, Fc)
    _, face, invz = ora.render_frame(mesh, K, T, H, W, want_faces=True, want_invz=True)
    face, invz = face.ravel(), invz.ravel().astype(np.float64)
    p = np.asarray(probs, dtype=np.float32).reshape(H * W, -1).astype(np.float64)
    c = p.shape[1]
    ys, xs = np.mgrid[0:H, 0:W]
    xs, ys = xs.ravel().astype(np.float64), ys.ravel().astype(np.float64)
    fx, fy, cx, cy = [float(v) for v in np.asarray(K, dtype=np.float64)]
    R = np.asarray(T, dtype=np.float64).reshape(4, 4)[:3, :3]
    ray = np.stack([(xs - cx) / fx, (ys - cy) / fy, np.ones_like(xs)], 1) @ R.T  # world direction
    Vd = V.astype(np.float64)
    f = np.maximum(face, 0)
    n = np.cross(Vd[Fc[f, 1]] - Vd[Fc[f, 0]], Vd[Fc[f, 2]] - Vd[Fc[f, 0]])
    cos = np.abs((n * ray).sum(1)) / (np.linalg.norm(n, axis=1) * np.linalg.norm(ray, axis=1))
    depth = np.where(face >= 0, 1.0 / np.where(invz > 0, invz, 1.0), 0.0) / 4.0
    ent = -(p * np.log(np.maximum(p, P_MIN))).sum(1) / np.log(c) if c > 1 else np.zeros(H * W)
    top = np.sort(p, axis=1)[:, ::-1]
    margin = top[:, 0] - (top[:, 1] if c > 1 else 0.0)
    border = np.minimum(np.minimum(xs, ys), np.minimum(W - 1 - xs, H - 1 - ys)) / (min(W, H) / 2.0)
    X = np.stack([cos, depth, ent, margin, border], 1)
    X[face < 0] = 0.0
    return X, face


def targets(probs, rows, labels):
    """y = 1 where the pixel's first arg max equals its row's fused label,
    0 elsewhere (and for background pixels)."""
    p = np.asarray(probs, dtype=np.float32).reshape(len(rows), -1)
    am = np.argmax(p, axis=1)
    rows = np.asarray(rows)
    lab = np.where(rows >= 0, np.asarray(labels)[np.maximum(rows, 0)], -1)
    return ((rows >= 0) & (am == lab)).astype(np.float64)
