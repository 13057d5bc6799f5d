"""Thin ctypes binding of liblabelfuse.so (include/labelfuse.h).

Every function here has the name of the C entry point it calls and only
marshals arguments: device buffers are passed as PyTorch CUDA tensors (or raw
integer addresses), the stream as a ``torch.cuda.Stream`` (default: the
current stream).  A non-OK status raises :class:`LabelFuseError` carrying
``sm_last_error()``.  There is no fallback: if the library is missing or was
not built, :func:`lib` raises.

A C entry point cannot see how large a buffer behind a pointer is, so the
binding checks every tensor argument before the call: contiguous, on the side
the call reads it from (CUDA, or host memory for ``sm_fuse_render_host``), and
at least as many bytes as the call reads or writes through it.  A violation
raises :class:`LabelFuseError` with ``SM_ERR_INVALID_ARG`` and nothing is
enqueued, so a wrong shape cannot make a kernel touch memory outside the
tensor.  Raw integer addresses are passed through unchecked.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblabelfuse.so")

SM_RULE = {"sum": 0, "logsum": 1, "maxsum": 2, "vote": 3}
SM_WEIGHT = {"pixel": 0, "image": 1}
SM_DTYPE = {"f32": 0, "bf16": 1, "fp8_e4m3": 2}
SM_KERNEL = {"project": 0, "raster": 1, "resolve": 2, "count": 3, "scatter": 4, "normalise": 5, "render": 6,
             "queue": 7, "conf": 8}
SM_OK = 0
SM_ERR_INVALID_ARG = 1
SM_ERR_INTERNAL = 6
SM_MAX_CLASSES = 254
SYMBOLS = ["sm_mesh_upload", "sm_fuse_frames", "sm_normalise", "sm_render_labels", "sm_render_idmap", "sm_reset",
           "sm_read_state", "sm_load_state", "sm_check", "sm_num_rows", "sm_num_classes", "sm_mesh_free",
           "sm_status_string", "sm_last_error", "sm_profile_enable", "sm_profile_read", "sm_render_rows_noalloc",
           "sm_fuse_render_host", "sm_host_alloc", "sm_host_free", "sm_device_alloc", "sm_device_free", "sm_set_weight_mix", "sm_texel_res_from_gamma",
           "sm_autotune_batch", "sm_fuse_frames_weighted", "sm_conf_features", "sm_conf_targets", "sm_conf_forward",
           "sm_conf_train_step", "sm_set_queue_shape", "sm_fuse_scenes", "sm_conf_weights",
           "sm_set_launch_frames", "sm_fuse_frames_confident", "sm_conf_train_step_indexed"]
SM_CONF_FEATURES = 5
SM_CONF_PARAMS = 1281
SM_NOALLOC_MAX_PIXELS = 1572864
SM_NOALLOC_MAX_FRAMES = 1024
SM_DEVICE_COMPRESSIBLE = 1


class SceneFrames(ctypes.Structure):
    """sm_scene_frames: one scene's frames for sm_fuse_scenes."""
    _fields_ = [("mesh", ctypes.c_void_p), ("d_probs", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("d_scale", ctypes.c_void_p), ("d_K", ctypes.c_void_p), ("d_cam_to_world", ctypes.c_void_p),
                ("N", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("d_idmap_out", ctypes.c_void_p)]


class LabelFuseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Loads liblabelfuse.so (build it with ``paper_2111_11103_gb300._build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2111_11103_gb300._build`")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sig = {
            "sm_mesh_upload": [P, i64, P, i64, P, i32, i32, i32, P, ctypes.POINTER(P)],
            "sm_fuse_frames": [P, P, i32, P, P, P, i32, i32, i32, P, P],
            "sm_normalise": [P, P, P, P],
            "sm_render_labels": [P, P, P, i32, i32, i32, P, P, P],
            "sm_render_idmap": [P, P, i64, P, P],
            "sm_reset": [P, P],
            "sm_read_state": [P, P, P, P],
            "sm_load_state": [P, P, P, P],
            "sm_check": [P, P],
            "sm_mesh_free": [P],
            "sm_profile_enable": [P, i32],
            "sm_render_rows_noalloc": [P, i64, P, i64, P, P, i32, i32, i32, P, P],
            "sm_fuse_render_host": [P, P, i32, P, P, P, i32, i32, i32, P, P],
            "sm_profile_read": [P, i32, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)],
            "sm_host_alloc": [ctypes.c_uint64, ctypes.POINTER(P)],
            "sm_host_free": [P],
            "sm_device_alloc": [i32, ctypes.c_uint64, i32, ctypes.POINTER(P), ctypes.POINTER(i32)],
            "sm_device_free": [P],
            "sm_set_weight_mix": [P, ctypes.c_float],
            "sm_texel_res_from_gamma": [P, P, P, i32, i32, i32, ctypes.c_float, P, P, P],
            "sm_autotune_batch": [P, P, i32, P, P, P, i32, i32, i32, ctypes.POINTER(i32), P],
            "sm_fuse_frames_weighted": [P, P, i32, P, P, P, i32, i32, i32, P, P, P],
            "sm_fuse_frames_confident": [P, P, i32, P, P, P, i32, i32, i32, P, P, P, P],
            "sm_conf_features": [P, P, i32, P, P, P, i32, i32, i32, P, P, P],
            "sm_conf_targets": [P, P, i32, P, P, i64, P, P],
            "sm_conf_forward": [P, P, i64, P, P],
            "sm_conf_train_step": [P, P, P, i64, ctypes.c_float, P, P, P],
            "sm_conf_train_step_indexed": [P, P, P, i64, P, i64, ctypes.c_float, P, P, P],
            "sm_set_queue_shape": [P, i32, i32, i32, i32, i32, i32],
            "sm_fuse_scenes": [P, i32, P],
            "sm_conf_weights": [P, P, i32, P, P, P, i32, i32, i32, P, P, P, P],
            "sm_set_launch_frames": [P, i32, i32, i32],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.sm_num_rows.argtypes = [P]
        L.sm_num_rows.restype = i64
        L.sm_num_classes.argtypes = [P]
        L.sm_num_classes.restype = i32
        L.sm_status_string.argtypes = [ctypes.c_int]
        L.sm_status_string.restype = ctypes.c_char_p
        L.sm_last_error.argtypes = []
        L.sm_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int):
    if status != SM_OK:
        raise LabelFuseError(status, lib().sm_last_error().decode() or lib().sm_status_string(status).decode())


def _arg(t, name: str, nbytes: int = 0, host: bool = False):
    """Address of a buffer argument after the checks described above: a
    tensor must be contiguous, a CUDA tensor (a CPU tensor if host), and hold
    at least nbytes.  None and raw integer addresses pass through."""
    if t is None or isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise LabelFuseError(SM_ERR_INVALID_ARG, f"{name} is not contiguous")
    if bool(t.is_cuda) == host:
        raise LabelFuseError(SM_ERR_INVALID_ARG, f"{name} must be a {'host (CPU)' if host else 'CUDA'} tensor")
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise LabelFuseError(SM_ERR_INVALID_ARG, f"{name} holds {have} bytes; the call needs {nbytes}")
    return t.data_ptr()


_ESIZE = {0: 4, 1: 2, 2: 1}  # bytes per stored probability: F32, BF16, FP8 E4M3


def _classes(mesh) -> int:
    """Classes of the mesh (0 for a NULL handle: the library rejects it)."""
    return max(0, int(lib().sm_num_classes(mesh))) if mesh else 0


def _frames_args(mesh, probs, dt: int, scale, K, cam_to_world, N: int, H: int, W: int, host: bool = False):
    """Checked addresses of the predictions, scales and cameras of N frames."""
    n, npix = max(0, int(N)), max(0, int(H)) * max(0, int(W))
    return (_arg(probs, "probs", n * npix * _classes(mesh) * _ESIZE.get(dt, 1), host),
            _arg(scale, "scale", 4 * n * npix, host),
            _arg(K, "K", 32 * n, host),
            _arg(cam_to_world, "cam_to_world", 128 * n, host))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _enum(table, v):
    return table[v] if isinstance(v, str) else int(v)


def sm_mesh_upload(vertices, faces, texel_res, n_classes: int, rule="sum", weight="pixel", stream=None) -> int:
    """Uploads a mesh; returns the opaque handle (an int).  vertices: V x 3
    float32 CUDA tensor; faces: F x 3 int32; texel_res: F int32 or None."""
    h = ctypes.c_void_p()
    V = int(vertices.shape[0]) if vertices is not None else 0
    F = int(faces.shape[0]) if faces is not None else 0
    _check(lib().sm_mesh_upload(_arg(vertices, "vertices", 12 * V), V, _arg(faces, "faces", 12 * F),
                                F, _arg(texel_res, "texel_res", 4 * F), int(n_classes),
                                _enum(SM_RULE, rule), _enum(SM_WEIGHT, weight), _stream(stream), ctypes.byref(h)))
    return h.value


def sm_fuse_frames(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, idmap_out=None,
                   stream=None):
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W)
    _check(lib().sm_fuse_frames(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                                _arg(idmap_out, "idmap_out", 4 * max(0, N * H * W)), _stream(stream)))


def sm_normalise(mesh: int, dist_out=None, labels_out=None, stream=None):
    n_x = max(0, sm_num_rows(mesh)) if mesh else 0
    _check(lib().sm_normalise(mesh, _arg(dist_out, "dist_out", 4 * n_x * _classes(mesh)),
                              _arg(labels_out, "labels_out", 4 * n_x), _stream(stream)))


def sm_render_labels(mesh: int, K, cam_to_world, N: int, H: int, W: int, labels_out, idmap_out=None, stream=None):
    n = max(0, N * H * W)
    _check(lib().sm_render_labels(mesh, _arg(K, "K", 32 * max(0, N)), _arg(cam_to_world, "cam_to_world", 128 * max(0, N)),
                                  int(N), int(H), int(W), _arg(labels_out, "labels_out", n),
                                  _arg(idmap_out, "idmap_out", 4 * n), _stream(stream)))


def sm_render_idmap(mesh: int, idmap, n_pixels: int, labels_out, stream=None):
    n = max(0, int(n_pixels))
    _check(lib().sm_render_idmap(mesh, _arg(idmap, "idmap", 4 * n), int(n_pixels), _arg(labels_out, "labels_out", n),
                                 _stream(stream)))


def sm_fuse_render_host(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, labels_out,
                        stream=None):
    """Fuse + normalise + render with HOST tensors (pin them for overlap)."""
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W, host=True)
    _check(lib().sm_fuse_render_host(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                                     _arg(labels_out, "labels_out", max(0, N * H * W), host=True), _stream(stream)))


def sm_set_weight_mix(mesh: int, alpha: float):
    _check(lib().sm_set_weight_mix(mesh, float(alpha)))


def sm_texel_res_from_gamma(mesh: int, K, cam_to_world, N: int, H: int, W: int, gamma: float, texel_res_out,
                            area_out=None, stream=None):
    # the outputs hold one value per triangle; the triangle count is not
    # visible through the handle, so only their placement is checked
    _check(lib().sm_texel_res_from_gamma(mesh, _arg(K, "K", 32 * max(0, N)),
                                         _arg(cam_to_world, "cam_to_world", 128 * max(0, N)), int(N), int(H), int(W),
                                         float(gamma), _arg(area_out, "area_out"), _arg(texel_res_out, "texel_res_out"),
                                         _stream(stream)))


def sm_autotune_batch(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, stream=None) -> int:
    """Chooses the frames per launch for H x W frames by timing; returns it."""
    best = ctypes.c_int32(0)
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W)
    _check(lib().sm_autotune_batch(mesh, p, dt, sc, k, t, int(N), int(H), int(W), ctypes.byref(best),
                                   _stream(stream)))
    return best.value


def sm_set_launch_frames(mesh: int, H: int, W: int, frames: int):
    """Frames per launch of the two-stream path for H x W frames (0: default)."""
    _check(lib().sm_set_launch_frames(mesh, int(H), int(W), int(frames)))


def sm_set_queue_shape(mesh: int, H: int, W: int, frames_per_batch: int, lookahead: int = 1, raster_rounds: int = 1,
                       scatter_tiles: int = 32):
    """Shape of the work-queue fusion for H x W frames; frames_per_batch = 0
    selects the two-stream path for this mesh."""
    _check(lib().sm_set_queue_shape(mesh, int(H), int(W), int(frames_per_batch), int(lookahead), int(raster_rounds),
                                    int(scatter_tiles)))


def sm_fuse_scenes(scenes, stream=None):
    """Fuses several scenes' frames, each into its own mesh (one call).
    scenes: (mesh, probs, dtype, scale, K, cam_to_world, N, H, W, idmap_out)
    per scene, with the arguments of sm_fuse_frames."""
    arr = (SceneFrames * max(1, len(scenes)))()
    for i, (mesh, probs, dtype, scale, K, T, N, H, W, idm) in enumerate(scenes):
        dt = _enum(SM_DTYPE, dtype)
        p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, T, N, H, W)
        arr[i] = SceneFrames(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                             _arg(idm, "idmap_out", 4 * max(0, N * H * W)))
    _check(lib().sm_fuse_scenes(arr if scenes else None, len(scenes), _stream(stream)))


def sm_fuse_frames_weighted(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, weights,
                            idmap_out=None, stream=None):
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W)
    n = max(0, N * H * W)
    _check(lib().sm_fuse_frames_weighted(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                                         _arg(weights, "weights", 4 * n), _arg(idmap_out, "idmap_out", 4 * n),
                                         _stream(stream)))


def sm_fuse_frames_confident(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, params,
                             w_out=None, idmap_out=None, stream=None):
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W)
    n = max(0, N * H * W)
    _check(lib().sm_fuse_frames_confident(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                                          _arg(params, "params", 4 * SM_CONF_PARAMS), _arg(w_out, "w_out", 4 * n),
                                          _arg(idmap_out, "idmap_out", 4 * n), _stream(stream)))


def sm_conf_features(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, feat_out, rows_out,
                     stream=None):
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W)
    n = max(0, N * H * W)
    _check(lib().sm_conf_features(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                                  _arg(feat_out, "feat_out", 4 * SM_CONF_FEATURES * n), _arg(rows_out, "rows_out", 4 * n),
                                  _stream(stream)))


def sm_conf_weights(mesh: int, probs, dtype, scale, K, cam_to_world, N: int, H: int, W: int, params, w_out, rows_out,
                    stream=None):
    dt = _enum(SM_DTYPE, dtype)
    p, sc, k, t = _frames_args(mesh, probs, dt, scale, K, cam_to_world, N, H, W)
    n = max(0, N * H * W)
    _check(lib().sm_conf_weights(mesh, p, dt, sc, k, t, int(N), int(H), int(W),
                                 _arg(params, "params", 4 * SM_CONF_PARAMS), _arg(w_out, "w_out", 4 * n),
                                 _arg(rows_out, "rows_out", 4 * n), _stream(stream)))


def sm_conf_targets(mesh: int, probs, dtype, scale, rows, n_pixels: int, target_out, stream=None):
    dt = _enum(SM_DTYPE, dtype)
    n = max(0, int(n_pixels))
    _check(lib().sm_conf_targets(mesh, _arg(probs, "probs", n * _classes(mesh) * _ESIZE.get(dt, 1)), dt,
                                 _arg(scale, "scale", 4 * n), _arg(rows, "rows", 4 * n), int(n_pixels),
                                 _arg(target_out, "target_out", 4 * n), _stream(stream)))


def sm_conf_forward(params, feat, n: int, w_out, stream=None):
    m = max(0, int(n))
    _check(lib().sm_conf_forward(_arg(params, "params", 4 * SM_CONF_PARAMS), _arg(feat, "feat", 4 * SM_CONF_FEATURES * m),
                                 int(n), _arg(w_out, "w_out", 4 * m), _stream(stream)))


def sm_conf_train_step(params, feat, target, n: int, lr: float, grad_out, loss_out, stream=None):
    m = max(0, int(n))
    _check(lib().sm_conf_train_step(_arg(params, "params", 4 * SM_CONF_PARAMS),
                                    _arg(feat, "feat", 4 * SM_CONF_FEATURES * m), _arg(target, "target", 4 * m), int(n),
                                    float(lr), _arg(grad_out, "grad_out", 4 * SM_CONF_PARAMS),
                                    _arg(loss_out, "loss_out", 4), _stream(stream)))


def sm_conf_train_step_indexed(params, feat, target, n_obs: int, idx, m: int, lr: float, grad_out, loss_out,
                               stream=None):
    """One training step on the minibatch of observations idx[0..m) (int64, device)."""
    no, mm = max(0, int(n_obs)), max(0, int(m))
    if idx is not None and not isinstance(idx, int) and str(idx.dtype) != "torch.int64":
        raise LabelFuseError(SM_ERR_INVALID_ARG, "idx must be int64")
    _check(lib().sm_conf_train_step_indexed(_arg(params, "params", 4 * SM_CONF_PARAMS),
                                            _arg(feat, "feat", 4 * SM_CONF_FEATURES * no), _arg(target, "target", 4 * no),
                                            int(n_obs), _arg(idx, "idx", 8 * mm), int(m), float(lr),
                                            _arg(grad_out, "grad_out", 4 * SM_CONF_PARAMS), _arg(loss_out, "loss_out", 4),
                                            _stream(stream)))


def sm_host_alloc(nbytes: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().sm_host_alloc(int(nbytes), ctypes.byref(p)))
    return p.value


def sm_host_free(p: int):
    _check(lib().sm_host_free(p))


class _HostBlock:
    """Owns one sm_host_alloc block; freed when the last tensor viewing it dies."""

    def __init__(self, nbytes: int):
        self.ptr = sm_host_alloc(nbytes)
        self.nbytes = nbytes

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().sm_host_free(self.ptr)
            self.ptr = None


def pinned_empty(shape, dtype):
    """Uninitialised CPU tensor in page-locked memory from sm_host_alloc (one
    block, copied to the device at the host link's full rate).  The memory is
    released with the tensor."""
    import math
    import torch
    shape = tuple(int(d) for d in shape)
    nbytes = max(1, math.prod(shape)) * torch.empty((), dtype=dtype).element_size()
    block = _HostBlock(nbytes)
    buf = (ctypes.c_uint8 * nbytes).from_address(block.ptr)
    buf._block = block  # the block lives as long as the buffer, which the tensor keeps
    return torch.frombuffer(buf, dtype=torch.uint8).view(dtype)[: math.prod(shape)].view(shape)


def sm_device_alloc(device: int, nbytes: int, compressible: bool = True) -> tuple[int, bool]:
    """(pointer, whether the block is compressible) of nbytes of device memory."""
    p = ctypes.c_void_p()
    comp = ctypes.c_int32(0)
    _check(lib().sm_device_alloc(int(device), int(nbytes), SM_DEVICE_COMPRESSIBLE if compressible else 0,
                                 ctypes.byref(p), ctypes.byref(comp)))
    return p.value, bool(comp.value)


def sm_device_free(p: int):
    _check(lib().sm_device_free(p))


_TYPESTR = {"torch.int32": "<i4", "torch.uint8": "|u1", "torch.float32": "<f4", "torch.int64": "<i8",
            "torch.int8": "|i1", "torch.bfloat16": "<V2", "torch.float16": "<f2"}


class _DeviceBlock:
    """Owns one sm_device_alloc block and exposes it as a CUDA array; the
    tensor made from it keeps it alive, and the block is freed with the last
    reference (sm_device_free waits for the device to be idle)."""

    def __init__(self, device: int, shape, dtype, compressible: bool):
        import math
        import torch
        self.ptr = None
        n = math.prod(shape)
        esize = torch.empty((), dtype=dtype).element_size()
        self.ptr, self.compressed = sm_device_alloc(device, max(1, n) * esize, compressible)
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": _TYPESTR[str(dtype)],
                                         "data": (self.ptr, False), "version": 2, "strides": None}

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().sm_device_free(self.ptr)
            self.ptr = None


def device_empty(shape, dtype, device=None, compressible: bool = True):
    """Uninitialised CUDA tensor in memory from sm_device_alloc: compressible
    where the GPU offers it (for row maps and label images, whose runs of equal
    values the memory system stores compressed).  The memory is released with
    the tensor; releasing a compressible block waits for the device to be idle,
    so let no such tensor die while a stream is being captured into a graph."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if dev.type != "cuda":
        raise ValueError("device_empty: a CUDA device is required")
    if str(dtype) not in _TYPESTR or dtype == torch.bfloat16:
        raise ValueError(f"device_empty: unsupported dtype {dtype}")
    shape = tuple(int(d) for d in shape)
    block = _DeviceBlock(dev.index if dev.index is not None else torch.cuda.current_device(), shape, dtype,
                         compressible)
    t = torch.as_tensor(block, device=dev)
    if t.data_ptr() != block.ptr:
        raise LabelFuseError(SM_ERR_INTERNAL, "device_empty: the tensor does not view the block")
    t.lf_compressed = block.compressed  # whether the memory is compressible
    return t


def sm_reset(mesh: int, stream=None):
    _check(lib().sm_reset(mesh, _stream(stream)))


def sm_read_state(mesh: int, acc_out=None, cnt_out=None, stream=None):
    n_x = max(0, sm_num_rows(mesh)) if mesh else 0
    _check(lib().sm_read_state(mesh, _arg(acc_out, "acc_out", 4 * n_x * _classes(mesh)),
                               _arg(cnt_out, "cnt_out", 4 * n_x), _stream(stream)))


def sm_load_state(mesh: int, acc, cnt, stream=None):
    n_x = max(0, sm_num_rows(mesh)) if mesh else 0
    _check(lib().sm_load_state(mesh, _arg(acc, "acc", 4 * n_x * _classes(mesh)), _arg(cnt, "cnt", 4 * n_x),
                               _stream(stream)))


def sm_check(mesh: int, stream=None):
    _check(lib().sm_check(mesh, _stream(stream)))


def sm_num_rows(mesh: int) -> int:
    return int(lib().sm_num_rows(mesh))


def sm_num_classes(mesh: int) -> int:
    return int(lib().sm_num_classes(mesh))


def sm_mesh_free(mesh: int):
    _check(lib().sm_mesh_free(mesh))


def sm_status_string(status: int) -> str:
    return lib().sm_status_string(int(status)).decode()


def sm_last_error() -> str:
    return lib().sm_last_error().decode()


def sm_render_rows_noalloc(vertices, faces, K, cam_to_world, N: int, H: int, W: int, idmap_out, stream=None):
    """Row maps (triangle per pixel) of N frames without any device allocation;
    for callers whose device memory is owned elsewhere (see labelfuse.h)."""
    import contextlib
    import torch
    V = int(vertices.shape[0]) if vertices is not None else 0
    F = int(faces.shape[0]) if faces is not None else 0
    n = max(0, int(N))
    # the library runs the call on the device that holds the output: take
    # that device's current stream unless one is given
    on_dev = isinstance(idmap_out, torch.Tensor) and idmap_out.is_cuda
    with (torch.cuda.device(idmap_out.device) if on_dev else contextlib.nullcontext()):
        _render_rows_noalloc(vertices, V, faces, F, K, cam_to_world, N, H, W, idmap_out, n, stream)


def _render_rows_noalloc(vertices, V, faces, F, K, cam_to_world, N, H, W, idmap_out, n, stream):
    _check(lib().sm_render_rows_noalloc(_arg(vertices, "vertices", 12 * V), V, _arg(faces, "faces", 12 * F), F,
                                        _arg(K, "K", 32 * n), _arg(cam_to_world, "cam_to_world", 128 * n), int(N),
                                        int(H), int(W), _arg(idmap_out, "idmap_out", 4 * max(0, N * H * W)),
                                        _stream(stream)))


def sm_profile_enable(mesh: int, on: bool = True):
    _check(lib().sm_profile_enable(mesh, 1 if on else 0))


def sm_profile_read(mesh: int, kernel) -> tuple[int, float]:
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(lib().sm_profile_read(mesh, _enum(SM_KERNEL, kernel), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value
