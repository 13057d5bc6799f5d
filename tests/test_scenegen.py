"""The seeded input generators: sizes, determinism, the face classes of
patch-aligned grids, and that patch-agnostic coarse grids really put
triangles across class boundaries (what the coarse-mesh study relies on)."""
import numpy as np
import pytest
import torch

import scenegen as sg


def test_paper_room_sizes_and_determinism():
    a = sg.paper_room(target_faces=60_000)
    b = sg.paper_room(target_faces=60_000)
    assert abs(len(a.faces) - 60_000) <= 0.01 * 60_000
    assert np.array_equal(a.faces, b.faces) and np.array_equal(a.vertices, b.vertices)
    assert np.array_equal(a.face_gt, b.face_gt)
    assert a.face_gt.min() >= 0 and a.face_gt.max() < a.n_classes
    for F in (100_000, 20_000, 5_000):
        c = sg.paper_room(target_faces=F, aligned=False)
        assert abs(len(c.faces) - F) <= 0.03 * F


def test_aligned_grid_triangles_stay_inside_one_patch():
    """Each triangle's three vertices lie in the patch of its class (closed
    patch boxes), for a patch-aligned grid."""
    s = sg.paper_room(target_faces=20_000)
    r = s.rects[0]  # the floor, gridded first
    pu, pv = r.classes.shape
    tri = s.vertices[s.faces].astype(np.float64)  # F x 3 x 3
    on_floor = np.all(np.abs(tri[..., 2] - r.origin[2]) < 1e-6, axis=1)
    first = int(np.argmin(on_floor))  # the floor is gridded first: its triangles lead
    t = tri[:first]
    u = (t[..., 0] - r.origin[0]) / np.linalg.norm(r.eu)
    v = (t[..., 1] - r.origin[1]) / np.linalg.norm(r.ev)
    iu = np.floor(u.mean(1) * pu).astype(int).clip(0, pu - 1)
    iv = np.floor(v.mean(1) * pv).astype(int).clip(0, pv - 1)
    lo_u, hi_u = iu / pu - 1e-9, (iu + 1) / pu + 1e-9
    lo_v, hi_v = iv / pv - 1e-9, (iv + 1) / pv + 1e-9
    assert np.all((u >= lo_u[:, None]) & (u <= hi_u[:, None]) & (v >= lo_v[:, None]) & (v <= hi_v[:, None]))
    assert np.array_equal(s.face_gt[:first], r.classes[iu, iv])


def test_coarse_unaligned_grid_straddles_patches():
    """A 5k-triangle patch-agnostic grid has triangles whose vertices lie in
    different class patches; its classes are those of the centroid's patch."""
    s = sg.paper_room(target_faces=5_000, aligned=False)
    r = s.rects[0]
    pu, pv = r.classes.shape
    tri = s.vertices[s.faces].astype(np.float64)
    first = int(np.argmin(np.all(np.abs(tri[..., 2] - r.origin[2]) < 1e-6, axis=1)))
    t = tri[:first]
    u = (t[..., 0] - r.origin[0]) / np.linalg.norm(r.eu)
    v = (t[..., 1] - r.origin[1]) / np.linalg.norm(r.ev)
    pu_idx = np.floor(np.clip(u, 0, 1 - 1e-12) * pu).astype(int)
    pv_idx = np.floor(np.clip(v, 0, 1 - 1e-12) * pv).astype(int)
    straddle = (pu_idx.min(1) != pu_idx.max(1)) | (pv_idx.min(1) != pv_idx.max(1))
    assert straddle.mean() > 0.3


def _covered(scene, p, tol=1e-9):
    """Whether point p lies on one of the scene's rectangles."""
    for r in scene.rects:
        n = np.cross(r.eu, r.ev)
        if abs(np.dot(p - r.origin, n)) > tol * np.linalg.norm(n):
            continue
        a = np.dot(p - r.origin, r.eu) / np.dot(r.eu, r.eu)
        b = np.dot(p - r.origin, r.ev) / np.dot(r.ev, r.ev)
        if 0 <= a <= 1 and 0 <= b <= 1:
            return True
    return False


def test_apartment_sizes_and_determinism():
    a = sg.apartment(target_faces=400_000)
    b = sg.apartment(target_faces=400_000)
    assert abs(len(a.faces) - 400_000) <= 0.01 * 400_000
    assert np.array_equal(a.faces, b.faces) and np.array_equal(a.vertices, b.vertices)
    assert np.array_equal(a.face_gt, b.face_gt)
    assert len(a.rects) == 6 + 4 * 3 + 4 * 20 * 5   # shell, 4 wall halves with doors, furniture
    assert a.face_gt.min() >= 0 and a.face_gt.max() < a.n_classes
    assert a.vertices[:, 0].max() <= 12.0 and a.vertices[:, 1].max() <= 10.0 and a.vertices[:, 2].max() <= 3.0


def test_apartment_doors_are_open_and_walls_closed():
    """Every neighbouring pair of rooms is joined by a 0.9 x 2.1 m door in the
    middle of its shared wall; the rest of that wall and the lintel are solid."""
    a = sg.apartment(target_faces=50_000)
    for centre, along in [((6.0, 2.5), (0, 1)), ((6.0, 7.5), (0, 1)), ((3.0, 5.0), (1, 0)), ((9.0, 5.0), (1, 0))]:
        c = np.array([centre[0], centre[1], 1.0])
        e = np.array([along[0], along[1], 0.0])
        assert not _covered(a, c)                                  # the door is open
        assert not _covered(a, c + 0.4 * e) and not _covered(a, c - 0.4 * e)
        assert _covered(a, c + 0.6 * e) and _covered(a, c - 0.6 * e)   # wall beside the door
        assert _covered(a, c + np.array([0.0, 0.0, 1.5]))          # lintel above it (z = 2.5)


def test_apartment_poses_stay_in_their_rooms():
    cams = sg.apartment_poses(400)
    assert cams.K.shape == (400, 4) and cams.cam_to_world.shape == (400, 4, 4)
    pos = cams.cam_to_world[:, :3, 3]
    for k in range(4):
        seg = pos[k * 100:(k + 1) * 100]
        x0, y0 = (k % 2) * 6.0, (k // 2) * 5.0
        assert np.all(seg[:, 0] >= x0 + 0.5 - 1e-9) and np.all(seg[:, 0] <= x0 + 5.5 + 1e-9)
        assert np.all(seg[:, 1] >= y0 + 0.5 - 1e-9) and np.all(seg[:, 1] <= y0 + 4.5 + 1e-9)
        assert np.allclose(seg[:, 2], 1.5)
    assert sg.apartment_poses(0).K.shape == (0, 4)


def test_oracle_sees_through_a_door(ora):
    """Rendered with the oracle from room (0, 0), facing the door to room (1, 0)
    head-on: pixels through the opening see triangles beyond the internal wall
    (x > 6 m), pixels beside it see the wall itself (x = 6 m)."""
    a = sg.apartment(target_faces=50_000)
    mesh = ora.Mesh(a.vertices, a.faces)
    T = sg._look_pose(np.array([4.5, 2.5, 1.0]), 0.0, 0.0, 0.0)   # 1.5 m before the door, looking +x
    K = np.array([40.0, 40.0, 31.5, 23.5])
    _, face = ora.render_frame(mesh, K, T, 48, 64, want_faces=True)
    x = a.vertices[a.faces].astype(np.float64)[..., 0].mean(1)    # triangle centroids' x
    # rows 4-12 cross the wall plane at z <= 1.73 m, inside the 2.1 m opening and
    # above every box (<= 1.2 m tall), so nothing of the first room is in the way
    centre = face[4:12, 28:36]                                     # through the 0.9 m opening
    assert np.all(centre >= 0) and np.all(x[centre] > 6.0 + 1e-6)
    side = face[4:12, 0:4]                                         # 0.75 m or more beside the door
    assert np.all(side >= 0) and np.allclose(x[side], 6.0)


def test_structured_recipe_errors_follow_view_difficulty():
    """The "structured" recipe: the error rate grows with the grazing angle,
    the depth beyond 2 m and the nearness to the border; the confuser class
    is never the true class; a frame's predictions are reproducible and
    wrong (arg max = confuser) far more often on hard pixels than on easy ones."""
    n = 128
    z = torch.full((n, n), 1.0, dtype=torch.float64)
    c1 = torch.ones((n, n), dtype=torch.float64)
    easy = sg.structured_error_rate(z, c1, n, n)
    assert float(easy[n // 2, n // 2]) == 0.0
    assert float(sg.structured_error_rate(z, c1 * 0.3, n, n)[n // 2, n // 2]) == pytest.approx(1.8 * 0.49)  # grazing
    assert float(sg.structured_error_rate(z * 6, c1, n, n)[n // 2, n // 2]) == pytest.approx(0.8)  # far
    assert float(easy[0, n // 2]) == pytest.approx(0.8)                                  # on the border
    assert float(easy[12, n // 2]) == pytest.approx(0.4)
    assert float(sg.structured_error_rate(z * 6, c1 * 0.3, n, n)[0, 0]) == 0.95          # capped
    H, W = 48, 64
    for c in (4, 20, 21, 40):
        gt = torch.arange(c)
        assert not torch.any(sg.confuser_class(gt, c) == gt)
    scene, cams = sg.paper_room(target_faces=20_000), sg.random_walk_poses(3, H=H, W=W, fx=58.0, fy=58.0,
                                                                             cx=31.5, cy=23.5)
    p1 = sg.predictions(scene, cams, "structured")
    assert torch.equal(p1, sg.predictions(scene, cams, "structured"))
    gt, depth, cosang = sg.ray_cast(scene, cams.K[0], cams.cam_to_world[0], H, W)
    assert torch.equal(gt, sg.ray_cast_classes(scene, cams.K[0], cams.cam_to_world[0], H, W))
    rate = sg.structured_error_rate(depth, cosang, H, W)
    wrong = (p1[0].argmax(-1) == sg.confuser_class(gt, scene.n_classes)) & (gt >= 0)
    hard, soft = rate > 0.5, (rate < 0.1) & (gt >= 0)
    assert hard.any() and soft.any()
    assert wrong[hard].float().mean() > 0.4 > 0.15 > wrong[soft].float().mean()
