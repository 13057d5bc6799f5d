"""Label-fusion oracle: plain, slow CPU reference of the method (arXiv 2111.11103).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and the two share no code.

The arithmetic lives in ``oracle.c`` (binary64 accumulation; the renderer's
integer decisions are taken in binary32 with a fixed operation order, so that
row maps are comparable bit for bit).  This module only compiles it and
marshals numpy arrays.  Which passage of the paper each function follows is
stated beside it in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RULES = {"sum": 0, "logsum": 1, "maxsum": 2, "vote": 3}
WEIGHTS = {"pixel": 0, "image": 1}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so with gcc (no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            L.ora_texel_count.restype = i64
            L.ora_texel_count.argtypes = [i64]
            L.ora_texel_id.restype = i64
            L.ora_texel_id.argtypes = [i64, i64]
            L.ora_texel_cell.restype = None
            L.ora_texel_cell.argtypes = [i32, ctypes.c_float, ctypes.c_float, P, P]
            L.ora_uv_origin.restype = i32
            L.ora_uv_origin.argtypes = [P, P, P]
            L.ora_row_offsets.restype = i64
            L.ora_row_offsets.argtypes = [P, i64, P]
            L.ora_projection.restype = None
            L.ora_projection.argtypes = [P, P, P]
            L.ora_render_frame.restype = i64
            L.ora_render_frame.argtypes = [P, i64, P, i64, P, P, P, P, P, i32, i32, P, P, P]
            L.ora_phi.restype = None
            L.ora_phi.argtypes = [i32, P, i32, P]
            L.ora_frame_weights.restype = None
            L.ora_frame_weights.argtypes = [i32, ctypes.c_double, P, i64, i64, P, P]
            L.ora_accumulate.restype = None
            L.ora_accumulate.argtypes = [i32, i64, P, P, P, i32, P, P]
            L.ora_normalise.restype = None
            L.ora_normalise.argtypes = [i32, P, P, i64, i32, P, P]
            L.ora_render_labels.restype = None
            L.ora_render_labels.argtypes = [P, i64, P, P]
            L.ora_fuse_sequence.restype = ctypes.c_int
            L.ora_fuse_sequence.argtypes = [P, i64, P, i64, P, P, P, i64, P, P, P, i32, i32, i32, i32, i32,
                                            i32, ctypes.c_double, i32, P, P, P]
            L.ora_visible_area.restype = ctypes.c_int
            L.ora_visible_area.argtypes = [P, i64, P, i64, P, P, i32, i32, i32, i32, P]
            L.ora_texel_res_from_gamma.restype = None
            L.ora_texel_res_from_gamma.argtypes = [P, i64, ctypes.c_float, P]
            L.ora_render_sequence.restype = ctypes.c_int
            L.ora_render_sequence.argtypes = [P, i64, P, i64, P, P, P, P, P, i32, i32, i32, i32, P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- texels
def texel_count(s: int) -> int:
    """|X_t| = (s^2 + s) / 2 (Sec. 3.1)."""
    return int(lib().ora_texel_count(int(s)))


def texel_id(i: int, j: int) -> int:
    """Texel identifier of cell (i, j): T(i + j) + j (Eq. idtexel, read as a bijection)."""
    return int(lib().ora_texel_id(int(i), int(j)))


def texel_cell(s: int, u: float, v: float) -> tuple[int, int]:
    i = ctypes.c_int32()
    j = ctypes.c_int32()
    lib().ora_texel_cell(int(s), float(u), float(v), ctypes.byref(i), ctypes.byref(j))
    return i.value, j.value


def uv_origin(p0, p1, p2) -> int:
    """Local index of the vertex with the interior angle closest to 90 degrees (Sec. 3.1)."""
    a, b, c = (np.ascontiguousarray(p, dtype=np.float32) for p in (p0, p1, p2))
    return int(lib().ora_uv_origin(_p(a), _p(b), _p(c)))


def uv_origins(vertices, faces) -> np.ndarray:
    V = np.asarray(vertices, dtype=np.float32)
    Fc = np.asarray(faces, dtype=np.int64)
    return np.array([uv_origin(V[f[0]], V[f[1]], V[f[2]]) for f in Fc], dtype=np.int32)


def row_offsets(F: int, s=None) -> tuple[np.ndarray, int]:
    """Row offsets id_t (F+1 entries) and n_x (Sec. 3.3.2)."""
    s = _c(s, np.int32)
    out = np.zeros(F + 1, dtype=np.int64)
    n_x = lib().ora_row_offsets(_p(s), int(F), _p(out))
    return out, int(n_x)


def projection(K, T) -> np.ndarray:
    K = _c(K, np.float64)
    T = _c(T, np.float64)
    A = np.zeros(12, dtype=np.float32)
    lib().ora_projection(_p(K), _p(T), _p(A))
    return A


# --------------------------------------------------------------------------- mesh
class Mesh:
    """Host copy of a mesh with its texel layout (s, uv origins, row offsets)."""

    def __init__(self, vertices, faces, texel_res=None):
        self.V = np.ascontiguousarray(vertices, dtype=np.float32).reshape(-1, 3)
        self.faces = np.ascontiguousarray(faces, dtype=np.int32).reshape(-1, 3)
        self.F = int(self.faces.shape[0])
        self.s = None if texel_res is None else np.ascontiguousarray(texel_res, dtype=np.int32)
        if self.s is not None and np.any(self.s > 1):
            self.origin = uv_origins(self.V, self.faces)
        else:
            self.origin = None
        self.id_t, self.n_x = row_offsets(self.F, self.s)


def render_frame(mesh: Mesh, K, T, H: int, W: int, want_faces: bool = False, want_invz: bool = False):
    """Row map (H x W int32, -1 = background) of one frame (Sec. 3.3.1); optionally
    also the winning triangle per pixel and its interpolated 1/z."""
    K = _c(K, np.float64)
    T = _c(T, np.float64)
    idmap = np.empty((H, W), dtype=np.int32)
    faces = np.empty((H, W), dtype=np.int32) if want_faces else None
    invz = np.empty((H, W), dtype=np.float32) if want_invz else None
    n = lib().ora_render_frame(_p(mesh.V), mesh.V.shape[0], _p(mesh.faces), mesh.F, _p(mesh.s), _p(mesh.origin),
                               _p(mesh.id_t), _p(K), _p(T), int(H), int(W), _p(idmap), _p(faces), _p(invz))
    if n < 0:
        raise MemoryError("oracle render_frame")
    out = (idmap,) + ((faces,) if want_faces else ()) + ((invz,) if want_invz else ())
    return out if len(out) > 1 else idmap


def render_sequence(mesh: Mesh, K, T, H: int, W: int, nthreads: int = 1) -> np.ndarray:
    K = _c(np.asarray(K).reshape(-1, 4), np.float64)
    T = _c(np.asarray(T).reshape(-1, 16), np.float64)
    N = K.shape[0]
    out = np.empty((N, H, W), dtype=np.int32)
    rc = lib().ora_render_sequence(_p(mesh.V), mesh.V.shape[0], _p(mesh.faces), mesh.F, _p(mesh.s),
                                   _p(mesh.origin), _p(mesh.id_t), _p(K), _p(T), N, int(H), int(W),
                                   int(nthreads), _p(out))
    if rc:
        raise MemoryError("oracle render_sequence")
    return out


# --------------------------------------------------------------------------- fusion
def phi(rule: str, p) -> np.ndarray:
    p = _c(p, np.float32)
    out = np.zeros(p.shape[-1], dtype=np.float64)
    lib().ora_phi(RULES[rule], _p(p), p.shape[-1], _p(out))
    return out


def frame_weights(weight: str, idmap, n_x: int, alpha: float = 1.0) -> np.ndarray:
    """Per-pixel weights of one frame: w^(P) = 1, or (1 - alpha) + alpha / n
    with n = pixels of the frame on the same row (alpha = 1: w^(I))."""
    idmap = _c(idmap, np.int32).ravel()
    counts = np.zeros(max(n_x, 1), dtype=np.int64)
    w = np.empty(idmap.size, dtype=np.float64)
    lib().ora_frame_weights(WEIGHTS[weight], float(alpha), _p(idmap), idmap.size, int(n_x), _p(counts), _p(w))
    return w


def accumulate(rule: str, rows, probs, n_x: int, weights=None, A=None, cnt=None):
    """A[l] += w * phi(p), cnt[l] += 1 over a list of observations (binary64)."""
    rows = _c(rows, np.int32).ravel()
    probs = _c(probs, np.float32).reshape(rows.size, -1)
    c = probs.shape[1]
    if A is None:
        A = np.zeros((n_x, c), dtype=np.float64)
    if cnt is None:
        cnt = np.zeros(n_x, dtype=np.int64)
    weights = _c(weights, np.float64)
    lib().ora_accumulate(RULES[rule], rows.size, _p(rows), _p(weights), _p(probs), c, _p(A), _p(cnt))
    return A, cnt


def fuse_frames(rule: str, weight: str, idmaps, probs, n_x: int, A=None, cnt=None):
    """Fuses frames whose row maps are already known, in frame order."""
    idmaps = _c(idmaps, np.int32)
    N = idmaps.shape[0]
    probs = _c(probs, np.float32).reshape(N, -1, probs.shape[-1])
    for i in range(N):
        w = frame_weights(weight, idmaps[i], n_x)
        A, cnt = accumulate(rule, idmaps[i].ravel(), probs[i], n_x, weights=w, A=A, cnt=cnt)
    return A, cnt


def fuse_sequence(mesh: Mesh, K, T, probs, rule: str, weight: str, nthreads: int = 1, want_idmaps: bool = False,
                  alpha: float = 1.0):
    """Renders and fuses all frames: returns (A, cnt[, idmaps]).  alpha mixes
    the image weight (weight == "image"): w = (1 - alpha) + alpha / n."""
    K = _c(np.asarray(K).reshape(-1, 4), np.float64)
    T = _c(np.asarray(T).reshape(-1, 16), np.float64)
    probs = _c(probs, np.float32)
    N, H, W, c = probs.shape
    A = np.zeros((mesh.n_x, c), dtype=np.float64)
    cnt = np.zeros(mesh.n_x, dtype=np.int64)
    idm = np.empty((N, H, W), dtype=np.int32) if want_idmaps else None
    rc = lib().ora_fuse_sequence(_p(mesh.V), mesh.V.shape[0], _p(mesh.faces), mesh.F, _p(mesh.s), _p(mesh.origin),
                                 _p(mesh.id_t), mesh.n_x, _p(K), _p(T), _p(probs), N, H, W, c, RULES[rule],
                                 WEIGHTS[weight], float(alpha), int(nthreads), _p(A), _p(cnt), _p(idm))
    if rc:
        raise MemoryError("oracle fuse_sequence")
    return (A, cnt, idm) if want_idmaps else (A, cnt)


def visible_area(vertices, faces, K, T, H: int, W: int, nthreads: int = 1) -> np.ndarray:
    """a_t: per triangle, the most pixels it is visible on in any one frame."""
    V = _c(vertices, np.float32).reshape(-1, 3)
    Fc = _c(faces, np.int32).reshape(-1, 3)
    K = _c(np.asarray(K).reshape(-1, 4), np.float64)
    T = _c(np.asarray(T).reshape(-1, 16), np.float64)
    area = np.zeros(Fc.shape[0], dtype=np.int64)
    if lib().ora_visible_area(_p(V), V.shape[0], _p(Fc), Fc.shape[0], _p(K), _p(T), K.shape[0], int(H), int(W),
                              int(nthreads), _p(area)):
        raise MemoryError("oracle visible_area")
    return area


def texel_res_from_gamma(area, gamma: float) -> np.ndarray:
    """s_t = max(1, ceil(gamma sqrt(a_t))) in binary32 (Sec. 3.1)."""
    area = _c(area, np.int64)
    s = np.empty(area.size, dtype=np.int32)
    lib().ora_texel_res_from_gamma(_p(area), area.size, float(gamma), _p(s))
    return s


def normalise(rule: str, A, cnt):
    """L1-normalised distributions and arg-max labels (-1 for unseen rows)."""
    A = _c(A, np.float64)
    cnt = _c(cnt, np.int64)
    n_x, c = A.shape
    dist = np.empty_like(A)
    labels = np.empty(n_x, dtype=np.int32)
    lib().ora_normalise(RULES[rule], _p(A), _p(cnt), n_x, c, _p(dist), _p(labels))
    return dist, labels


def render_labels(idmaps, labels) -> np.ndarray:
    idmaps = _c(idmaps, np.int32)
    labels = _c(labels, np.int32)
    out = np.empty(idmaps.shape, dtype=np.uint8)
    lib().ora_render_labels(_p(idmaps), idmaps.size, _p(labels), _p(out))
    return out
