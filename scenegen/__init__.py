"""Seeded synthetic inputs shaped like the paper's indoor RGB-D sequences.

This module makes the inputs that both the CUDA library and the oracle consume:
procedural room meshes with a ground-truth class per triangle, camera
trajectories (intrinsics + camera-to-world poses) and noisy softmax
"network predictions".  It holds none of the fusion method's arithmetic: the
per-pixel ground truth used to shape a prediction comes from an analytic ray
cast against the scene's rectangles (a stand-in for what a segmentation
network looks at), not from the method's triangle raster.

Recipes (all seed-fixed):

* ``tiny_room``: cube room [-1, 1]^3, the four side walls each gridded into
  16 x 16 quads (2 triangles each: 2,048 triangles); ground-truth class = wall
  index (c = 4).  ``circle_poses``: 8 cameras on a circle of radius 0.5 m at
  the room centre, looking outward; 64 x 48 pixels, fx = fy = 58, cx = 32,
  cy = 24.  Predictions: softmax(3 onehot(gt) + N(0, 1)).
* ``paper_room``: 6 x 5 x 3 m room with 20 axis-aligned boxes on the floor
  (sides U(0.3, 1.5) m, height U(0.3, 1.2) m); every rectangle cut into
  <= 0.5 m patches with a Zipf(1) class over c = 40 classes and gridded into
  quads whose size is chosen so the mesh has the requested triangle count
  (500k +- 1 %).  ``random_walk_poses``: camera at 1.5 m, xy from an
  Ornstein-Uhlenbeck velocity walk (stationary speed sd 0.3 m/s, 30 fps) kept
  >= 0.5 m from the walls, smooth yaw walk, pitch around -15 deg (sd 5 deg),
  roll around 0 (sd 2 deg); 640 x 480, fx = fy = 577.6, cx = 319.5, cy = 239.5.
  Predictions: softmax(2.5 onehot(gt) + field + N(0, 0.5^2)), with ``field`` a
  per-frame, per-class 11 x 8 control grid of N(0, 1.2^2) bilinearly upsampled.
* ``apartment``: four such rooms (6 x 5 x 3 m each, 20 boxes each) in a 2 x 2
  layout, the two crossing internal walls opened by a 0.9 x 2.1 m door in each
  half, gridded to ~4M triangles (the learned-confidence configuration).
  ``apartment_poses``: one ``random_walk_poses`` segment per room.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

BASE_SEED = 2111111030


@dataclasses.dataclass
class Rect:
    origin: np.ndarray  # (3,)
    eu: np.ndarray      # (3,) edge vector
    ev: np.ndarray      # (3,) edge vector
    classes: np.ndarray  # (pu, pv) class per patch


@dataclasses.dataclass
class Scene:
    vertices: np.ndarray   # V x 3 float32 (world, metres, z up)
    faces: np.ndarray      # F x 3 int32
    face_gt: np.ndarray    # F int32 ground-truth class
    rects: list            # analytic description for ground-truth ray casts
    n_classes: int


@dataclasses.dataclass
class Cameras:
    K: np.ndarray          # N x 4 float64 (fx, fy, cx, cy)
    cam_to_world: np.ndarray  # N x 4 x 4 float64 row-major
    H: int
    W: int


# --------------------------------------------------------------------------- meshes
def _grid_rect(rect: Rect, nu: int, nv: int, v_base: int):
    a = np.arange(nu + 1, dtype=np.float64) / nu
    b = np.arange(nv + 1, dtype=np.float64) / nv
    A, B = np.meshgrid(a, b, indexing="ij")
    P = rect.origin[None, None, :] + A[..., None] * rect.eu[None, None, :] + B[..., None] * rect.ev[None, None, :]
    verts = P.reshape(-1, 3)
    idx = np.arange((nu + 1) * (nv + 1)).reshape(nu + 1, nv + 1) + v_base
    v00 = idx[:-1, :-1].ravel()
    v10 = idx[1:, :-1].ravel()
    v01 = idx[:-1, 1:].ravel()
    v11 = idx[1:, 1:].ravel()
    tris = np.stack([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 1).reshape(-1, 3)
    pu, pv = rect.classes.shape
    # the class of the patch under each quad's centre (the same as quad // (nu / pu)
    # when the grid refines the patches; a grid that ignores them cuts across patches)
    qa = np.minimum(((np.arange(nu) + 0.5) * pu / nu).astype(np.int64), pu - 1)
    qb = np.minimum(((np.arange(nv) + 0.5) * pv / nv).astype(np.int64), pv - 1)
    cls = rect.classes[qa[:, None], qb[None, :]].ravel()
    gt = np.repeat(cls, 2)
    return verts, tris, gt


def _build(rects, quads, n_classes):
    Vs, Fs, Gs = [], [], []
    base = 0
    for r, (nu, nv) in zip(rects, quads):
        v, f, g = _grid_rect(r, nu, nv, base)
        Vs.append(v)
        Fs.append(f)
        Gs.append(g)
        base += v.shape[0]
    return Scene(np.concatenate(Vs).astype(np.float32), np.concatenate(Fs).astype(np.int32),
                 np.concatenate(Gs).astype(np.int32), rects, n_classes)


def tiny_room() -> Scene:
    """Cube room [-1,1]^3: four side walls, 16 x 16 quads each, class = wall index."""
    o = np.array
    rects = [
        Rect(o([1.0, -1.0, -1.0]), o([0.0, 2.0, 0.0]), o([0.0, 0.0, 2.0]), np.full((1, 1), 0)),   # x = +1
        Rect(o([-1.0, -1.0, -1.0]), o([0.0, 2.0, 0.0]), o([0.0, 0.0, 2.0]), np.full((1, 1), 1)),  # x = -1
        Rect(o([-1.0, 1.0, -1.0]), o([2.0, 0.0, 0.0]), o([0.0, 0.0, 2.0]), np.full((1, 1), 2)),   # y = +1
        Rect(o([-1.0, -1.0, -1.0]), o([2.0, 0.0, 0.0]), o([0.0, 0.0, 2.0]), np.full((1, 1), 3)),  # y = -1
    ]
    return _build(rects, [(16, 16)] * 4, 4)


def _zipf_classes(rng, shape, n_classes):
    p = 1.0 / np.arange(1, n_classes + 1)
    p /= p.sum()
    return rng.choice(n_classes, size=shape, p=p)


def paper_room(seed: int = BASE_SEED + 1, target_faces: int = 500_000, n_boxes: int = 20,
               n_classes: int = 40, size=(6.0, 5.0, 3.0), aligned: bool = True) -> Scene:
    """Procedural room with box furniture, ~target_faces triangles (+-1 %).
    aligned=False grids every rectangle without regard to its class patches
    (as a simplified reconstruction would): coarse grids then have triangles
    that straddle class boundaries (about +-3 % of target_faces)."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = size
    o = np.array
    geo = [  # (origin, eu, ev) of every rectangle
        (o([0.0, 0.0, 0.0]), o([Lx, 0.0, 0.0]), o([0.0, Ly, 0.0])),  # floor
        (o([0.0, 0.0, Lz]), o([Lx, 0.0, 0.0]), o([0.0, Ly, 0.0])),   # ceiling
        (o([0.0, 0.0, 0.0]), o([Lx, 0.0, 0.0]), o([0.0, 0.0, Lz])),  # y = 0
        (o([0.0, Ly, 0.0]), o([Lx, 0.0, 0.0]), o([0.0, 0.0, Lz])),   # y = Ly
        (o([0.0, 0.0, 0.0]), o([0.0, Ly, 0.0]), o([0.0, 0.0, Lz])),  # x = 0
        (o([Lx, 0.0, 0.0]), o([0.0, Ly, 0.0]), o([0.0, 0.0, Lz])),   # x = Lx
    ]
    geo += _boxes(rng, n_boxes, 0.0, 0.0, Lx, Ly)
    return _mesh_rects(_patch_rects(rng, geo, n_classes), target_faces, aligned, n_classes)


def _boxes(rng, n: int, x_lo: float, y_lo: float, Lx: float, Ly: float):
    """n axis-aligned boxes standing on the floor of the Lx x Ly area whose
    corner is (x_lo, y_lo): sides U(0.3, 1.5) m, height U(0.3, 1.2) m; the five
    visible rectangles of each (no bottom)."""
    o = np.array
    geo = []
    for _ in range(n):
        w, d = rng.uniform(0.3, 1.5, size=2)
        h = rng.uniform(0.3, 1.2)
        x0 = x_lo + rng.uniform(0.0, Lx - w)
        y0 = y_lo + rng.uniform(0.0, Ly - d)
        geo += [
            (o([x0, y0, h]), o([w, 0.0, 0.0]), o([0.0, d, 0.0])),      # top
            (o([x0, y0, 0.0]), o([w, 0.0, 0.0]), o([0.0, 0.0, h])),    # front
            (o([x0, y0 + d, 0.0]), o([w, 0.0, 0.0]), o([0.0, 0.0, h])),  # back
            (o([x0, y0, 0.0]), o([0.0, d, 0.0]), o([0.0, 0.0, h])),    # left
            (o([x0 + w, y0, 0.0]), o([0.0, d, 0.0]), o([0.0, 0.0, h])),  # right
        ]
    return geo


def _wall_with_door(start, along, length: float, height: float, door_w: float, door_h: float):
    """A vertical wall from `start` along the unit vector `along`, with a door
    opening of door_w x door_h centred on it: the part left of the door, the
    part right of it and the lintel above it."""
    z = np.array([0.0, 0.0, 1.0])
    side = 0.5 * (length - door_w)
    return [
        (start, along * side, z * height),
        (start + along * (side + door_w), along * side, z * height),
        (start + along * side + z * door_h, along * door_w, z * (height - door_h)),
    ]


def apartment(seed: int = BASE_SEED + 5, target_faces: int = 4_000_000, boxes_per_room: int = 20,
              n_classes: int = 40, room=(6.0, 5.0, 3.0), door=(0.9, 2.1), aligned: bool = True) -> Scene:
    """Four rooms of room[0] x room[1] x room[2] m in a 2 x 2 layout under one
    floor and ceiling, with the same furniture and class patches as
    ``paper_room``.  The two internal walls (x = room[0], y = room[1]) cross at
    the middle; each half of each has a door of door[0] x door[1] m at its
    centre, so every pair of neighbouring rooms is joined.  ~target_faces
    triangles (+-1 %)."""
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = room
    X, Y = 2 * Lx, 2 * Ly
    o = np.array
    ex, ey = o([1.0, 0.0, 0.0]), o([0.0, 1.0, 0.0])
    geo = [
        (o([0.0, 0.0, 0.0]), o([X, 0.0, 0.0]), o([0.0, Y, 0.0])),    # floor
        (o([0.0, 0.0, Lz]), o([X, 0.0, 0.0]), o([0.0, Y, 0.0])),     # ceiling
        (o([0.0, 0.0, 0.0]), o([X, 0.0, 0.0]), o([0.0, 0.0, Lz])),   # y = 0
        (o([0.0, Y, 0.0]), o([X, 0.0, 0.0]), o([0.0, 0.0, Lz])),     # y = Y
        (o([0.0, 0.0, 0.0]), o([0.0, Y, 0.0]), o([0.0, 0.0, Lz])),   # x = 0
        (o([X, 0.0, 0.0]), o([0.0, Y, 0.0]), o([0.0, 0.0, Lz])),     # x = X
    ]
    for y0 in (0.0, Ly):   # internal wall x = Lx, one door per room pair
        geo += _wall_with_door(o([Lx, y0, 0.0]), ey, Ly, Lz, door[0], door[1])
    for x0 in (0.0, Lx):   # internal wall y = Ly
        geo += _wall_with_door(o([x0, Ly, 0.0]), ex, Lx, Lz, door[0], door[1])
    for i in range(2):
        for j in range(2):
            geo += _boxes(rng, boxes_per_room, i * Lx, j * Ly, Lx, Ly)
    return _mesh_rects(_patch_rects(rng, geo, n_classes), target_faces, aligned, n_classes)


def _patch_rects(rng, geo, n_classes):
    """Rectangles cut into <= 0.5 m patches, each with a Zipf(1) class."""
    rects = []
    for org, eu, ev in geo:
        pu = max(1, math.ceil(np.linalg.norm(eu) / 0.5 - 1e-9))
        pv = max(1, math.ceil(np.linalg.norm(ev) / 0.5 - 1e-9))
        rects.append(Rect(org, eu, ev, _zipf_classes(rng, (pu, pv), n_classes)))
    return rects


def _mesh_rects(rects, target_faces: int, aligned: bool, n_classes: int) -> Scene:
    """Grids every rectangle into quads of one edge length chosen so that the
    mesh has about target_faces triangles: aligned grids refine each class
    patch (then +-1 quad-per-patch steps bring the count within 0.5 %),
    unaligned grids ignore the patches."""
    def quads_for(hq):
        out = []
        for r in rects:
            pu, pv = r.classes.shape
            if not aligned:
                out.append((max(1, int(round(np.linalg.norm(r.eu) / hq))), max(1, int(round(np.linalg.norm(r.ev) / hq)))))
                continue
            qu = max(1, int(round(np.linalg.norm(r.eu) / pu / hq)))
            qv = max(1, int(round(np.linalg.norm(r.ev) / pv / hq)))
            out.append((pu * qu, pv * qv))
        return out

    def nfaces(hq):
        return sum(2 * nu * nv for nu, nv in quads_for(hq))

    area = sum(np.linalg.norm(np.cross(r.eu, r.ev)) for r in rects)
    lo, hi = 0.2 * math.sqrt(2 * area / target_faces), 5.0 * math.sqrt(2 * area / target_faces)
    for _ in range(60):  # bisection on the quad edge length
        mid = 0.5 * (lo + hi)
        if nfaces(mid) > target_faces:
            lo = mid
        else:
            hi = mid
    hq = min((lo, hi), key=lambda q: abs(nfaces(q) - target_faces))
    if not aligned:
        return _build(rects, quads_for(hq), n_classes)
    per = [[nu // r.classes.shape[0], nv // r.classes.shape[1]] for r, (nu, nv) in zip(rects, quads_for(hq))]

    def total():
        return sum(2 * r.classes.shape[0] * q[0] * r.classes.shape[1] * q[1] for r, q in zip(rects, per))

    for _ in range(500):  # greedy +-1 quad-per-patch steps until within 0.5 %
        err = total() - target_faces
        if abs(err) <= 0.005 * target_faces:
            break
        best = None
        for ri, r in enumerate(rects):
            pu, pv = r.classes.shape
            for ax in (0, 1):
                step = -1 if err > 0 else 1
                q = list(per[ri])
                if q[ax] + step < 1:
                    continue
                q[ax] += step
                new_err = err + 2 * pu * pv * (q[0] * q[1] - per[ri][0] * per[ri][1])
                if best is None or abs(new_err) < best[0]:
                    best = (abs(new_err), ri, ax, step)
        if best is None or best[0] >= abs(err):
            break
        per[best[1]][best[2]] += best[3]
    quads = [(r.classes.shape[0] * q[0], r.classes.shape[1] * q[1]) for r, q in zip(rects, per)]
    return _build(rects, quads, n_classes)



# --------------------------------------------------------------------------- cameras
def _look_pose(pos, yaw, pitch, roll):
    """Camera-to-world 4x4 (camera x right, y down, z forward; world z up)."""
    cp, sp = math.cos(pitch), math.sin(pitch)
    cyw, syw = math.cos(yaw), math.sin(yaw)
    f = np.array([cp * cyw, cp * syw, sp])
    r = np.array([syw, -cyw, 0.0])
    d = np.cross(f, r)
    cr, sr = math.cos(roll), math.sin(roll)
    r2 = cr * r + sr * d
    d2 = -sr * r + cr * d
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = r2, d2, f, pos
    return T


def circle_poses(n: int = 8, radius: float = 0.5, H: int = 48, W: int = 64, fx: float = 58.0,
                 fy: float = 58.0, cx: float = 32.0, cy: float = 24.0) -> Cameras:
    """n cameras on a circle at the room centre, looking radially outward."""
    Ts = []
    for k in range(n):
        a = 2.0 * math.pi * k / n
        Ts.append(_look_pose(np.array([radius * math.cos(a), radius * math.sin(a), 0.0]), a, 0.0, 0.0))
    K = np.tile(np.array([fx, fy, cx, cy], dtype=np.float64), (n, 1))
    return Cameras(K, np.stack(Ts), H, W)


def random_walk_poses(n: int, seed: int = BASE_SEED + 1, size=(6.0, 5.0, 3.0), height: float = 1.5,
                      margin: float = 0.5, H: int = 480, W: int = 640, fx: float = 577.6, fy: float = 577.6,
                      cx: float = 319.5, cy: float = 239.5, fps: float = 30.0, origin=None) -> Cameras:
    """Smooth random-walk trajectory inside the room (see module docstring);
    origin: (x, y) of the room's corner if it is not at the world origin."""
    rng = np.random.default_rng(seed + 7919)
    dt = 1.0 / fps
    theta = 1.0  # 1/s mean reversion of the velocity
    lo = np.array([margin, margin])
    hi = np.array([size[0] - margin, size[1] - margin])
    p = rng.uniform(lo, hi)
    v = rng.normal(0.0, 0.3, size=2)
    yaw = rng.uniform(-math.pi, math.pi)
    yaw_rate = 0.0
    pitch_dev, roll_dev = 0.0, 0.0
    Ts = []
    for _ in range(n):
        pos = np.array([p[0], p[1], height]) if origin is None else np.array([origin[0] + p[0], origin[1] + p[1], height])
        T = _look_pose(pos, yaw, math.radians(-15.0) + pitch_dev, roll_dev)
        Ts.append(T)
        v += -theta * v * dt + 0.3 * math.sqrt(2 * theta * dt) * rng.normal(size=2)
        p = p + v * dt
        for a in range(2):  # reflect at the margins
            if p[a] < lo[a]:
                p[a] = 2 * lo[a] - p[a]
                v[a] = -v[a]
            if p[a] > hi[a]:
                p[a] = 2 * hi[a] - p[a]
                v[a] = -v[a]
        yaw_rate += -2.0 * yaw_rate * dt + 0.6 * math.sqrt(4.0 * dt) * rng.normal()
        yaw += yaw_rate * dt
        pitch_dev += -1.0 * pitch_dev * dt + math.radians(5.0) * math.sqrt(2 * dt) * rng.normal()
        roll_dev += -1.0 * roll_dev * dt + math.radians(2.0) * math.sqrt(2 * dt) * rng.normal()
    K = np.tile(np.array([fx, fy, cx, cy], dtype=np.float64), (n, 1))
    return Cameras(K, np.stack(Ts), H, W)


def apartment_poses(n: int, seed: int = BASE_SEED + 5, room=(6.0, 5.0, 3.0), **kw) -> Cameras:
    """n frames for ``apartment``: one random-walk segment per room (rooms in
    the order (0,0), (1,0), (0,1), (1,1), frames split as evenly as
    possible), each kept >= 0.5 m from that room's walls.  The segments are
    concatenated; fusion treats frames as independent observations."""
    parts = []
    for k in range(4):
        nk = n // 4 + (1 if k < n % 4 else 0)
        if nk:
            parts.append(random_walk_poses(nk, seed=seed + k, size=room, origin=((k % 2) * room[0], (k // 2) * room[1]),
                                           **kw))
    if not parts:
        return Cameras(np.zeros((0, 4)), np.zeros((0, 4, 4)), kw.get("H", 480), kw.get("W", 640))
    return Cameras(np.concatenate([c.K for c in parts]), np.concatenate([c.cam_to_world for c in parts]),
                   parts[0].H, parts[0].W)


# --------------------------------------------------------------------------- ground truth + predictions
def ray_cast_classes(scene: Scene, K, T, H: int, W: int, device="cpu", chunk: int = 65536) -> torch.Tensor:
    """Class of the nearest rectangle seen through every pixel centre (analytic
    ray cast against the scene's rectangles); -1 where nothing is hit."""
    return ray_cast(scene, K, T, H, W, device, chunk)[0]


def ray_cast(scene: Scene, K, T, H: int, W: int, device="cpu", chunk: int = 65536):
    """Analytic ray cast through every pixel centre: (class of the nearest
    rectangle, -1 where nothing is hit; its depth along the optical axis;
    |cos| of the angle between the viewing ray and the rectangle's normal),
    each H x W (depth and cos are 0 where nothing is hit)."""
    dev = torch.device(device)
    fx, fy, cx, cy = (float(x) for x in K)
    Tt = torch.as_tensor(np.asarray(T, dtype=np.float64), device=dev)
    ys, xs = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float64),
                            torch.arange(W, device=dev, dtype=torch.float64), indexing="ij")
    dc = torch.stack([(xs - cx) / fx, (ys - cy) / fy, torch.ones_like(xs)], -1).reshape(-1, 3)
    dirs = dc @ Tt[:3, :3].T
    C = Tt[:3, 3]
    O = torch.as_tensor(np.stack([r.origin for r in scene.rects]), device=dev)
    EU = torch.as_tensor(np.stack([r.eu for r in scene.rects]), device=dev)
    EV = torch.as_tensor(np.stack([r.ev for r in scene.rects]), device=dev)
    Nrm = torch.cross(EU, EV, dim=1)
    CO = C[None, :] - O
    tnum = -(CO * Nrm).sum(1)
    cu, cv = (CO * EU).sum(1), (CO * EV).sum(1)
    nu, nv = (EU * EU).sum(1), (EV * EV).sum(1)
    pus = torch.as_tensor([r.classes.shape[0] for r in scene.rects], device=dev)
    pvs = torch.as_tensor([r.classes.shape[1] for r in scene.rects], device=dev)
    offs = torch.as_tensor(np.cumsum([0] + [r.classes.size for r in scene.rects])[:-1], device=dev)
    flat = torch.as_tensor(np.concatenate([r.classes.ravel() for r in scene.rects]), device=dev)
    out = torch.empty(H * W, dtype=torch.int64, device=dev)
    depth = torch.zeros(H * W, dtype=torch.float64, device=dev)
    cosang = torch.zeros(H * W, dtype=torch.float64, device=dev)
    nn = torch.linalg.norm(Nrm, dim=1)
    for s in range(0, H * W, chunk):
        d = dirs[s:s + chunk]
        t = tnum[None, :] / (d @ Nrm.T)
        a = (cu[None, :] + t * (d @ EU.T)) / nu[None, :]
        b = (cv[None, :] + t * (d @ EV.T)) / nv[None, :]
        ok = (t > 1e-6) & (a >= 0) & (a < 1) & (b >= 0) & (b < 1) & torch.isfinite(t)
        t = torch.where(ok, t, torch.full_like(t, float("inf")))
        tmin, ridx = t.min(1)
        ai = a.gather(1, ridx[:, None])[:, 0]
        bi = b.gather(1, ridx[:, None])[:, 0]
        pu, pv = pus[ridx], pvs[ridx]
        iu = torch.minimum(torch.clamp((ai * pu).floor().long(), min=0), pu - 1)
        iv = torch.minimum(torch.clamp((bi * pv).floor().long(), min=0), pv - 1)
        cls = flat[offs[ridx] + iu * pv + iv]
        hit = torch.isfinite(tmin)
        out[s:s + chunk] = torch.where(hit, cls, torch.full_like(cls, -1))
        # the camera-space direction has z = 1, so the ray parameter is the depth
        depth[s:s + chunk] = torch.where(hit, tmin, torch.zeros_like(tmin))
        cs = ((d * Nrm[ridx]).sum(1)).abs() / (torch.linalg.norm(d, dim=1) * nn[ridx])
        cosang[s:s + chunk] = torch.where(hit, cs, torch.zeros_like(cs))
    return out.reshape(H, W), depth.reshape(H, W), cosang.reshape(H, W)


RECIPES = {
    # boost, i.i.d. noise sd, spatial field sd (0 = none)
    "tiny": (3.0, 1.0, 0.0),
    "paper": (2.5, 0.5, 1.2),
    "structured": (2.5, 0.5, 0.6),
}


def structured_error_rate(depth, cosang, H: int, W: int):
    """Probability that the "structured" recipe's prediction of a pixel is
    confidently wrong: it grows with the grazing angle (1 - |cos|), with the
    depth beyond 2 m and near the image border (within 24 pixels), as a
    segmentation network's errors do: 1.8 (1 - |cos|)^2 + 0.8 clamp((z - 2) /
    4) + 0.8 clamp(1 - d / 24) for depth z in m and border distance d in
    pixels, at most 0.95."""
    dev = depth.device
    ys, xs = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float64),
                            torch.arange(W, device=dev, dtype=torch.float64), indexing="ij")
    border = torch.minimum(torch.minimum(xs, ys), torch.minimum(W - 1 - xs, H - 1 - ys))
    r = (1.8 * (1.0 - cosang) ** 2 + 0.8 * ((depth - 2.0) / 4.0).clamp(0.0, 1.0)
         + 0.8 * (1.0 - border / 24.0).clamp(0.0, 1.0))
    return r.clamp(0.0, 0.95)


def confuser_class(gt: torch.Tensor, c: int) -> torch.Tensor:
    """The wrong class the "structured" recipe predicts for true class gt:
    (7 gt + 3) mod c, never gt for even c (7 gt + 3 = gt mod c would need
    6 gt = -3 mod c, odd against even); gt + 1 for odd c."""
    wrong = (7 * gt + 3) % c
    return torch.where(wrong == gt, (gt + 1) % c, wrong)


def predictions(scene: Scene, cams: Cameras, recipe: str = "paper", frames=None, seed: int = BASE_SEED,
                device="cpu", out: torch.Tensor | None = None, gt_out: torch.Tensor | None = None) -> torch.Tensor:
    """Softmax predictions (len(frames) x H x W x c float32, HWC) on ``device``.
    Recipes: "tiny" and "paper" (see the module docstring); "structured" adds
    confidently wrong predictions (a fixed confuser class per true class) at
    a rate that grows with the grazing angle, the depth and the nearness to
    the image border (structured_error_rate), for the learned confidence.

    gt_out, if given (len(frames) x H x W, any integer type), receives the
    ground-truth class of every pixel (-1: nothing hit).

    Frame i draws its noise from a generator seeded with (seed, i) only, so a
    frame's values do not depend on which other frames are generated with it
    (they do depend on the device: CPU and CUDA generators differ)."""
    boost, sd, field_sd = RECIPES[recipe]
    structured = recipe == "structured"
    dev = torch.device(device)
    frames = range(cams.K.shape[0]) if frames is None else frames
    frames = list(frames)
    H, W, c = cams.H, cams.W, scene.n_classes
    if out is None:
        out = torch.empty((len(frames), H, W, c), dtype=torch.float32, device=dev)
    for n, i in enumerate(frames):
        g = torch.Generator(device=dev)
        g.manual_seed((seed * 1_000_003 + i * 7_919) % (2 ** 63 - 1))
        gt, depth, cosang = ray_cast(scene, cams.K[i], cams.cam_to_world[i], H, W, device=dev)
        if gt_out is not None:
            gt_out[n] = gt
        logits = torch.randn((H, W, c), generator=g, device=dev, dtype=torch.float32) * sd
        if field_sd > 0:
            grid = torch.randn((1, c, 8, 11), generator=g, device=dev, dtype=torch.float32) * field_sd
            field = torch.nn.functional.interpolate(grid, size=(H, W), mode="bilinear", align_corners=True)
            logits += field[0].permute(1, 2, 0)
        onehot = torch.zeros((H, W, c), device=dev, dtype=torch.float32)
        valid = gt >= 0
        if structured:  # confidently wrong where the view is hard (grazing, far, border)
            u = torch.rand((H, W), generator=g, device=dev, dtype=torch.float64)
            wrong = valid & (u < structured_error_rate(depth, cosang, H, W))
            gt = torch.where(wrong, confuser_class(gt, c), gt)
        onehot[valid, gt[valid]] = boost
        logits += onehot
        out[n] = torch.softmax(logits, dim=-1)
    return out


def pixel_ground_truth(face_gt: np.ndarray, face_map: np.ndarray) -> np.ndarray:
    """Ground-truth class per pixel from a per-pixel triangle map (-1 = none)."""
    fm = np.asarray(face_map)
    out = np.full(fm.shape, -1, dtype=np.int32)
    m = fm >= 0
    out[m] = face_gt[fm[m]]
    return out
