"""Pins for the oracle's renderer (Sec. 3.3.1): hand-counted coverage, a
closed-form wall, brute-force ray-triangle casts on tiny meshes, the
near-plane reading and the texel ids of a subdivided triangle."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
IDENT = np.eye(4)


def _pixel_camera():
    """Identity pose and K = (1, 1, 0, 0): vertex (x, y, 1) projects to pixel (x, y)."""
    return np.array([1.0, 1.0, 0.0, 0.0]), IDENT


def _hand_cases():
    rows = []
    for line in open(os.path.join(GOLDEN, "hand_coverage.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        parts = line.split()
        name, nums, expect = parts[0], [float(x) for x in parts[1:-1]], int(parts[-1])
        rows.append((name, np.array(nums).reshape(-1, 2), expect))
    return rows


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c[0])
def test_hand_counted_coverage(ora, case):
    name, xy, expect = case
    V = np.concatenate([xy, np.ones((len(xy), 1))], 1)
    if len(xy) == 3:
        faces = np.array([[0, 1, 2]])
    else:
        faces = np.array([[0, 1, 2], [0, 2, 3]])
    K, T = _pixel_camera()
    mesh = ora.Mesh(V, faces)
    idmap = ora.render_frame(mesh, K, T, 16, 16)
    assert int((idmap >= 0).sum()) == expect
    if len(faces) == 2:
        # shared edge: each triangle alone, coverage disjoint and the union is the square
        cov = []
        for f in range(2):
            m1 = ora.Mesh(V, faces[f:f + 1])
            cov.append(ora.render_frame(m1, K, T, 16, 16) >= 0)
        assert not np.any(cov[0] & cov[1])
        assert int((cov[0] | cov[1]).sum()) == expect
        ys, xs = np.nonzero(cov[0] | cov[1])
        assert xs.min() == 0 and xs.max() == 7 and ys.min() == 0 and ys.max() == 7


def test_hand_counted_pixels_exact(ora):
    """The integer right triangle covers exactly {x>=0, y>=0, x+y<8}."""
    V = np.array([[0, 0, 1], [8, 0, 1], [0, 8, 1]], dtype=np.float64)
    K, T = _pixel_camera()
    idmap = ora.render_frame(ora.Mesh(V, [[0, 1, 2]]), K, T, 12, 12)
    ys, xs = np.mgrid[0:12, 0:12]
    assert np.array_equal(idmap >= 0, (xs + ys < 8))


@pytest.mark.parametrize("frac,expect_le", [(0.6, True), (0.4, False)])
def test_snap_rounds_to_nearest(ora, frac, expect_le):
    """Vertices snap to the nearest 1/256 pixel (Sec. 3.3.1 reading).  The legs
    of the right triangle (0,0), (a,0), (0,a) are a = 5 + frac/256 pixels:
    frac = 0.6 snaps the hypotenuse to 1281/256, so the six centres with
    x + y = 5 are inside (21 pixels); frac = 0.4 snaps it onto them (1280/256),
    where the bottom-right edge excludes them (15 pixels)."""
    a = 5 + frac / 256
    V = np.array([[0, 0, 1], [a, 0, 1], [0, a, 1]], dtype=np.float64)
    K, T = _pixel_camera()
    idmap = ora.render_frame(ora.Mesh(V, [[0, 1, 2]]), K, T, 10, 10)
    ys, xs = np.mgrid[0:10, 0:10]
    expect = (xs + ys <= 5) if expect_le else (xs + ys < 5)
    assert int(expect.sum()) == (21 if expect_le else 15)
    assert np.array_equal(idmap >= 0, expect)


def test_sequence_render_matches_frames(ora):
    """The threaded row-map renderer gives every frame's own row map, for one
    and for several threads."""
    import scenegen as sg
    sc = sg.tiny_room()
    cams = sg.circle_poses()
    mesh = ora.Mesh(sc.vertices, sc.faces)
    one = np.stack([ora.render_frame(mesh, cams.K[i], cams.cam_to_world[i], cams.H, cams.W)
                    for i in range(cams.K.shape[0])])
    assert len({one[i].tobytes() for i in range(len(one))}) == len(one)  # the views differ
    for nthreads in (1, 3):
        seq = ora.render_sequence(mesh, cams.K, cams.cam_to_world, cams.H, cams.W, nthreads=nthreads)
        assert np.array_equal(seq, one)


def test_closed_form_wall(ora):
    """A fronto-parallel wall at depth 2: the covered rectangle follows from the
    intrinsics (edges at x = 3.25, 13.25 and y = 2.5, 10.0; the bottom edge is
    not a top/left edge, so row 10 is excluded) and every covered pixel has
    1/z = 0.5 exactly."""
    V = np.array([[-1, -0.75, 2], [1, -0.75, 2], [1, 0.75, 2], [-1, 0.75, 2]], dtype=np.float64)
    K = np.array([10.0, 10.0, 8.25, 6.25])
    mesh = ora.Mesh(V, [[0, 1, 2], [0, 2, 3]])
    idmap, invz = ora.render_frame(mesh, K, IDENT, 14, 18, want_invz=True)
    ys, xs = np.mgrid[0:14, 0:18]
    expect = (xs >= 4) & (xs <= 13) & (ys >= 3) & (ys <= 9)
    assert np.array_equal(idmap >= 0, expect)
    assert np.all(invz[expect] == np.float32(0.5))


def test_depth_order_and_tie(ora):
    """Nearest wins; an exact depth tie goes to the lower triangle index."""
    near = [[0, 0, 1.0], [8, 0, 1.0], [0, 8, 1.0]]
    far = [[0, 0, 2.0], [16, 0, 2.0], [0, 16, 2.0]]    # same footprint at depth 2
    K, T = _pixel_camera()
    for order in ([0, 1], [1, 0]):
        tris = [near, far] if order == [0, 1] else [far, near]
        V = np.array(tris[0] + tris[1], dtype=np.float64)
        mesh = ora.Mesh(V, [[0, 1, 2], [3, 4, 5]])
        _, faces = ora.render_frame(mesh, K, T, 10, 10, want_faces=True)
        near_idx = order.index(0)
        assert np.all(faces[faces >= 0] == near_idx)
    # identical triangles listed twice: lower index wins everywhere
    V = np.array(near + near, dtype=np.float64)
    _, faces = ora.render_frame(ora.Mesh(V, [[0, 1, 2], [3, 4, 5]]), K, T, 10, 10, want_faces=True)
    assert np.all(faces[faces >= 0] == 0) and (faces >= 0).sum() == 36


def test_near_plane_drops_triangle(ora):
    """A triangle with a vertex at depth <= 0.05 is dropped whole (no clipping)."""
    K, T = _pixel_camera()
    V = np.array([[0, 0, 1.0], [8, 0, 1.0], [0, 8, 0.05]], dtype=np.float64)
    assert (ora.render_frame(ora.Mesh(V, [[0, 1, 2]]), K, T, 10, 10) >= 0).sum() == 0
    V[2, 2] = 0.0501
    assert (ora.render_frame(ora.Mesh(V, [[0, 1, 2]]), K, T, 200, 200) >= 0).sum() > 0


def test_degenerate_and_offscreen(ora):
    K, T = _pixel_camera()
    line = np.array([[0, 0, 1.0], [4, 4, 1.0], [8, 8, 1.0]])
    assert (ora.render_frame(ora.Mesh(line, [[0, 1, 2]]), K, T, 10, 10) >= 0).sum() == 0
    off = np.array([[-20, -20, 1.0], [-10, -20, 1.0], [-20, -10, 1.0]])
    assert (ora.render_frame(ora.Mesh(off, [[0, 1, 2]]), K, T, 10, 10) >= 0).sum() == 0
    behind = np.array([[0, 0, -1.0], [8, 0, -1.0], [0, 8, -1.0]])
    assert (ora.render_frame(ora.Mesh(behind, [[0, 1, 2]]), K, T, 10, 10) >= 0).sum() == 0


def _moller_trumbore(O, D, V0, V1, V2):
    """Ray/triangle distances (binary64) for rays D (P x 3) against triangles (R)."""
    e1, e2 = V1 - V0, V2 - V0
    pvec = np.cross(D[:, None, :], e2[None])
    det = (e1[None] * pvec).sum(-1)
    tvec = O[None, None, :] - V0[None]
    u = (tvec * pvec).sum(-1) / det
    qvec = np.cross(tvec, e1[None])
    v = (D[:, None, :] * qvec).sum(-1) / det
    t = (e2[None] * qvec).sum(-1) / det
    ok = (np.abs(det) > 1e-12) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
    return np.where(ok, t, np.inf)


def _seg_dist(P, A, B):
    AB = B - A
    t = np.clip(((P - A) * AB).sum(-1) / np.maximum((AB * AB).sum(-1), 1e-300), 0, 1)
    Q = A + t[..., None] * AB
    return np.sqrt(((P - Q) ** 2).sum(-1))


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_ray_cast(ora, seed):
    """Tiny random meshes (48 triangles, 32 x 24 pixels, random pose): the
    oracle's winning triangle equals an FP64 Moller-Trumbore ray cast through
    every pixel centre, except pixels within 2/256 px of a projected edge or
    within 1e-5 relative depth of the runner-up (listed, not failed)."""
    rng = np.random.default_rng(100 + seed)
    H, W = 24, 32
    K = np.array([30.0, 30.0, 15.5, 11.5])
    # random camera pose
    ang = rng.uniform(-np.pi, np.pi, 3)
    cz, sz = np.cos(ang[0]), np.sin(ang[0])
    cy_, sy_ = np.cos(ang[1]), np.sin(ang[1])
    cx_, sx_ = np.cos(ang[2]), np.sin(ang[2])
    R = (np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]]) @ np.array([[cy_, 0, sy_], [0, 1, 0], [-sy_, 0, cy_]])
         @ np.array([[1, 0, 0], [0, cx_, -sx_], [0, sx_, cx_]]))
    C = rng.normal(size=3)
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, C
    ntri = 48
    centres_c = np.stack([rng.uniform(-0.6, 0.6, ntri), rng.uniform(-0.5, 0.5, ntri), np.ones(ntri)], 1)
    centres_c *= rng.uniform(1.0, 4.0, ntri)[:, None]
    Vc = centres_c[:, None, :] + rng.normal(scale=0.35, size=(ntri, 3, 3)) * centres_c[:, None, 2:3]
    Vw = (Vc @ R.T + C).reshape(-1, 3).astype(np.float32).astype(np.float64)
    faces = np.arange(ntri * 3).reshape(-1, 3)
    mesh = ora.Mesh(Vw, faces)
    _, fmap = ora.render_frame(mesh, K, T, H, W, want_faces=True)

    # brute force in binary64 (camera frame)
    Vcam = ((Vw - C) @ R).reshape(ntri, 3, 3)
    ys, xs = np.mgrid[0:H, 0:W]
    D = np.stack([(xs - K[2]) / K[0], (ys - K[3]) / K[1], np.ones_like(xs, dtype=np.float64)], -1).reshape(-1, 3)
    tt = _moller_trumbore(np.zeros(3), D, Vcam[:, 0], Vcam[:, 1], Vcam[:, 2])
    valid_tri = np.all(Vcam[:, :, 2] > 0.05, axis=1)
    tt[:, ~valid_tri] = np.inf
    order = np.argsort(tt, axis=1)
    best = np.where(np.isfinite(tt[np.arange(len(D)), order[:, 0]]), order[:, 0], -1)
    t1 = tt[np.arange(len(D)), order[:, 0]]
    t2 = tt[np.arange(len(D)), order[:, 1]]
    # projected (unsnapped) vertices, pixel distance to every edge of every valid triangle
    proj = np.stack([K[0] * Vcam[..., 0] / Vcam[..., 2] + K[2], K[1] * Vcam[..., 1] / Vcam[..., 2] + K[3]], -1)
    Pp = np.stack([xs, ys], -1).reshape(-1, 1, 2).astype(np.float64)
    dmin = np.full(len(D), np.inf)
    for e in range(3):
        d = _seg_dist(Pp, proj[None, :, e], proj[None, :, (e + 1) % 3])
        d[:, ~valid_tri] = np.inf
        dmin = np.minimum(dmin, d.min(1))
    with np.errstate(invalid="ignore"):
        ambiguous = (dmin < 2.0 / 256) | (np.isfinite(t2) & (np.abs(t2 - t1) < 1e-5 * t1))
    got = fmap.ravel()
    bad = (got != best) & ~ambiguous
    assert not np.any(bad), f"{bad.sum()} mismatching pixels"
    assert (~ambiguous).sum() > 0.9 * H * W
    assert (best >= 0).sum() > 50  # the scene is actually visible


@pytest.mark.parametrize("flip", [False, True])
def test_texel_rows_on_subdivided_triangle(ora, flip):
    """A large triangle with s = 6 seen head-on, in both windings (one of them
    goes through the renderer's orientation fix-up): every one of its 21
    texels is hit (Fig. 3), the rows stay inside [id_t, id_t + 21), and each
    pixel's texel is the cell of its uv coordinates computed independently in
    binary64 from the face's own vertex order (u toward its second vertex
    after the uv origin, v toward its third)."""
    V = np.array([[0, 0, 1.0], [60, 0, 1.0], [0, 60, 1.0], [70, 70, 1.0], [75, 70, 1.0], [70, 75, 1.0]])
    tri = [0, 2, 1] if flip else [0, 1, 2]
    faces = np.array([[3, 4, 5], tri])
    s = np.array([1, 6], dtype=np.int32)
    mesh = ora.Mesh(V, faces, texel_res=s)
    assert mesh.n_x == 22 and list(mesh.id_t) == [0, 1, 22]
    K, T = _pixel_camera()
    idmap, fmap = ora.render_frame(mesh, K, T, 64, 64, want_faces=True)
    rows = idmap[fmap == 1]
    assert set(rows.tolist()) == set(range(1, 22))
    o = mesh.origin[1]
    assert o == 0  # right angle at the face's first vertex (V0) in both windings
    ys, xs = np.nonzero(fmap == 1)
    # barycentric coordinates in binary64 (affine: all depths equal)
    P0, P1, P2 = (V[tri[(o + k) % 3], :2] for k in range(3))
    M = np.stack([P1 - P0, P2 - P0], 1)
    uv = np.linalg.solve(M, (np.stack([xs, ys], 1) - P0).T).T   # weights of the 2nd and 3rd vertex
    u, v = uv[:, 0], uv[:, 1]
    i = np.minimum(np.floor(6 * u), 5).astype(int)
    j = np.minimum(np.floor(6 * v), 5 - i).astype(int)
    near_border = (np.abs(6 * u - np.round(6 * u)) < 1e-4) | (np.abs(6 * v - np.round(6 * v)) < 1e-4)
    expect = 1 + (i + j) * (i + j + 1) // 2 + j
    assert np.all((idmap[ys, xs] == expect) | near_border)
    assert (~near_border).sum() > 1000


def test_s1_equals_face_mode(ora):
    """At gamma = 0 (s = 1 everywhere) the row map equals the face map (Sec. 3.1)."""
    import scenegen as sg
    sc = sg.tiny_room()
    cams = sg.circle_poses()
    m0 = ora.Mesh(sc.vertices, sc.faces)
    m1 = ora.Mesh(sc.vertices, sc.faces, texel_res=np.ones(len(sc.faces), np.int32))
    for i in range(cams.K.shape[0]):
        a, fa = ora.render_frame(m0, cams.K[i], cams.cam_to_world[i], cams.H, cams.W, want_faces=True)
        b = ora.render_frame(m1, cams.K[i], cams.cam_to_world[i], cams.H, cams.W)
        assert np.array_equal(a, b) and np.array_equal(a, fa)
        assert np.all(a >= 0)  # tiny room: the walls fill every view
