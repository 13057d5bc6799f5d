"""Frame-sharded fusion over several processes (one GPU each).

Every fusion rule accumulates a sum over the frames that see a row (Sec. 3.2:
Eqs. sum and maxsum directly, Eq. mul in the log domain; the update of
Sec. 3.3.2 does not depend on the order of the frames).  So the frames of a
sequence can be split into disjoint ranges, each range fused on its own GPU
into its own accumulators, and one all-reduce (sum) of the accumulators and
observation counts gives every rank the state of the whole sequence.  Row
normalisation and render-back then run on every rank, render-back for its
own frames.

Host-side logic only: the fusion itself runs in the CUDA library
(``labelfuse``); the exchange is ``torch.distributed.all_reduce`` (NCCL on
GPUs, gloo on the CPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def frame_range(n_frames: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of this rank's frames: contiguous, sizes differing by at
    most one, in rank order, covering [0, n_frames) exactly once."""
    if world < 1 or not 0 <= rank < world or n_frames < 0:
        raise ValueError(f"bad shard: n_frames={n_frames}, rank={rank}, world={world}")
    base, extra = divmod(n_frames, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_state(acc: torch.Tensor, cnt: torch.Tensor, group=None) -> None:
    """Sums the accumulators (float32, n_x x c) and observation counts
    (int32, n_x) of all ranks, in place."""
    if acc.dtype != torch.float32 or cnt.dtype != torch.int32:
        raise TypeError("accumulators must be float32 and counts int32")
    dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM, group=group)


def complete_fusion(mesh: int, state=None, group=None) -> None:
    """After each rank has fused its own frames into the mesh: one all-reduce
    of the accumulators and counts, loaded back, so that every rank holds the
    whole sequence's state.  state: optional (acc, cnt) buffers to reuse.
    Enqueued on the current CUDA stream, which the collective follows."""
    from . import labelfuse as lf
    if state is None:
        import torch
        n_x, c = lf.sm_num_rows(mesh), lf.sm_num_classes(mesh)
        dev = torch.device("cuda", torch.cuda.current_device())
        state = (torch.empty((max(n_x, 1), c), dtype=torch.float32, device=dev),
                 torch.empty(max(n_x, 1), dtype=torch.int32, device=dev))
    acc, cnt = state
    lf.sm_read_state(mesh, acc, cnt)
    allreduce_state(acc, cnt, group)
    lf.sm_load_state(mesh, acc, cnt)


def fuse_sharded(mesh: int, probs, dtype, scale, K, cam_to_world, H: int, W: int, rank: int, world: int,
                 idmap_out=None, group=None, state=None) -> tuple[int, int]:
    """Fuses this rank's frames of the sequence (probs, scale, K, cam_to_world
    hold all N frames) into the mesh, then all-reduces the state so that every
    rank holds the whole sequence's accumulators.  idmap_out, if given,
    receives this rank's row maps.  state: optional (acc, cnt) buffers to
    reuse.  Everything is enqueued on the current CUDA stream, which the
    collective follows.  Returns the rank's frame range."""
    from . import labelfuse as lf
    n = int(K.shape[0])
    a, b = frame_range(n, rank, world)
    if b > a:
        lf.sm_fuse_frames(mesh, probs[a:b], dtype, None if scale is None else scale[a:b], K[a:b],
                          cam_to_world[a:b], b - a, H, W, idmap_out)
    if state is None:
        n_x, c = lf.sm_num_rows(mesh), lf.sm_num_classes(mesh)
        state = (torch.empty((max(n_x, 1), c), dtype=torch.float32, device=probs.device),
                 torch.empty(max(n_x, 1), dtype=torch.int32, device=probs.device))
    complete_fusion(mesh, state, group)
    return a, b
