"""Learned per-observation confidence, end to end: features of every pixel,
targets from a plain fusion (does the pixel's arg max agree with its row's
fused label?), gradient descent on the network, then fusion weighted by the
network's output.  Host-side orchestration of the C ABI (the features,
network, training steps and weighted fusion all run in the library)."""
from __future__ import annotations

import numpy as np
import torch

from . import labelfuse as lf


def init_params(seed: int = 0, scale: float = 0.2, device="cuda") -> torch.Tensor:
    rng = np.random.default_rng(seed)
    return torch.as_tensor(rng.normal(0.0, scale, lf.SM_CONF_PARAMS).astype(np.float32), device=device)


def train(mesh: int, probs, K, cam_to_world, H: int, W: int, steps: int = 200, lr: float = 1.0, seed: int = 0,
          batch: int | None = None, dtype="f32", scale=None):
    """Trains the network on the sequence's observations.  mesh: a mesh whose
    rule the targets come from; it is reset, fused (unweighted) and
    normalised here, and left in that state.  Returns (params, losses)."""
    lf.sm_reset(mesh)
    lf.sm_fuse_frames(mesh, probs, dtype, scale, K, cam_to_world, int(K.shape[0]), H, W)
    lf.sm_normalise(mesh)
    return train_on_labels(mesh, probs, K, cam_to_world, H, W, steps, lr, seed, batch, dtype, scale)


def train_on_labels(mesh: int, probs, K, cam_to_world, H: int, W: int, steps: int = 200, lr: float = 1.0,
                    seed: int = 0, batch: int | None = None, dtype="f32", scale=None):
    """Trains the network on the observations of the given frames, labelled
    by agreement with the mesh's current fused labels (the mesh must be
    normalised: e.g. a plain fusion of a whole sequence, of which these frames
    are a sample).  The mesh's state is left as it is.  Returns (params,
    losses)."""
    N, dev = int(K.shape[0]), probs.device
    feat = torch.empty((N, H, W, lf.SM_CONF_FEATURES), device=dev)
    rows = torch.empty((N, H, W), dtype=torch.int32, device=dev)
    lf.sm_conf_features(mesh, probs, dtype, scale, K, cam_to_world, N, H, W, feat, rows)
    y = torch.empty((N, H, W), device=dev)
    lf.sm_conf_targets(mesh, probs, dtype, scale, rows, N * H * W, y)
    sel = rows.reshape(-1) >= 0
    X, Y = feat.reshape(-1, lf.SM_CONF_FEATURES)[sel].contiguous(), y.reshape(-1)[sel].contiguous()
    params = init_params(seed, device=dev)
    grad = torch.empty(lf.SM_CONF_PARAMS, device=dev)
    loss = torch.empty(steps, device=dev)
    g = torch.Generator(device=dev).manual_seed(seed)
    for s in range(steps):
        if batch and batch < X.shape[0]:
            # the minibatch's indices are drawn here (random numbers are the
            # step's input); the step reads the observations where they lie
            idx = torch.randint(0, X.shape[0], (batch,), device=dev, generator=g)
            lf.sm_conf_train_step_indexed(params, X, Y, X.shape[0], idx, batch, lr, grad, loss[s:s + 1])
        else:
            lf.sm_conf_train_step(params, X, Y, X.shape[0], lr, grad, loss[s:s + 1])
    return params, loss.cpu().numpy()


def fuse_with_confidence(mesh: int, params, probs, K, cam_to_world, H: int, W: int, dtype="f32", scale=None,
                         idmap_out=None, w_out=None):
    """Fuses the frames into the mesh with each observation weighed by the
    network's confidence, one raster pass per frame (sm_fuse_frames_confident:
    per batch the raster, the features and network, then the weighted
    scatter).  w_out: optional N x H x W float32 tensor for the weights."""
    N = int(K.shape[0])
    lf.sm_fuse_frames_confident(mesh, probs, dtype, scale, K, cam_to_world, N, H, W, params, w_out, idmap_out)
    return w_out
