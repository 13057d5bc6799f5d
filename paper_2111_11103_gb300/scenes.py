"""Many independent scenes at once: each scene's fusion (its own mesh,
accumulators and frames) is enqueued on one of a few CUDA streams, so small
scenes that cannot fill the GPU alone run side by side.  Host-side
orchestration of the C ABI only; every step runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses

import torch


@dataclasses.dataclass
class SceneJob:
    mesh: int                    # handle from sm_mesh_upload
    probs: torch.Tensor          # N x H x W x c on the device
    K: torch.Tensor              # N x 4 intrinsics (float64)
    cam_to_world: torch.Tensor   # N x 16 poses (float64)
    H: int
    W: int
    dtype: str = "f32"
    scale: torch.Tensor | None = None
    idmap_out: torch.Tensor | None = None
    dist_out: torch.Tensor | None = None
    labels_out: torch.Tensor | None = None


_POOLS: dict = {}


def _pool(n: int) -> list:
    """n streams of the current device, created once and reused (so that a
    call can be captured into a CUDA graph after a first eager call)."""
    key = (torch.cuda.current_device(), n)
    if key not in _POOLS:
        _POOLS[key] = [torch.cuda.Stream() for _ in range(n)]
    return _POOLS[key]


def fuse_scenes_queued(jobs: list[SceneJob]) -> None:
    """Fuses (and, where an output is given, normalises) every scene with one
    sm_fuse_scenes call on the current stream: scenes that the work queue
    applies to share persistent launches (the library groups them by class
    count, storage type and rule); the others are fused one by one."""
    from . import labelfuse as lf
    if len({j.mesh for j in jobs}) != len(jobs):
        raise ValueError("a mesh may appear in one job only")
    if not jobs:
        return
    lf.sm_fuse_scenes([(j.mesh, j.probs, j.dtype, j.scale, j.K, j.cam_to_world, int(j.K.shape[0]), j.H, j.W,
                        j.idmap_out) for j in jobs])
    for j in jobs:
        if j.dist_out is not None or j.labels_out is not None:
            lf.sm_normalise(j.mesh, j.dist_out, j.labels_out)


def fuse_scenes(jobs: list[SceneJob], streams: int = 4) -> None:
    """Fuses (and, where an output is given, normalises) every scene; scene i
    runs on stream i % streams.  The streams start after the work already on
    the current stream and the current stream waits for all of them, so the
    call orders like one sequence of calls on the current stream, and it can
    be captured into a CUDA graph (after one eager call that creates the
    streams).  A mesh must appear in one job only."""
    from . import labelfuse as lf
    if len({j.mesh for j in jobs}) != len(jobs):
        raise ValueError("a mesh may appear in one job only")
    if not jobs:
        return
    cur = torch.cuda.current_stream()
    pool = _pool(max(1, min(streams, len(jobs))))
    for st in pool:
        st.wait_stream(cur)
    capturing = torch.cuda.is_current_stream_capturing()
    for i, j in enumerate(jobs):
        st = pool[i % len(pool)]
        n = int(j.K.shape[0])
        lf.sm_fuse_frames(j.mesh, j.probs, j.dtype, j.scale, j.K, j.cam_to_world, n, j.H, j.W, j.idmap_out, st)
        if j.dist_out is not None or j.labels_out is not None:
            lf.sm_normalise(j.mesh, j.dist_out, j.labels_out, st)
        if not capturing:  # (a graph keeps its tensors alive itself)
            # the caller's tensors were used on this job's stream
            for t in (j.probs, j.K, j.cam_to_world, j.scale, j.idmap_out, j.dist_out, j.labels_out):
                if t is not None:
                    t.record_stream(st)
    for st in pool:
        cur.wait_stream(st)
