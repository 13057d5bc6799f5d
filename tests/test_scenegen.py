"""The seeded input generators: sizes, determinism, the face classes of
patch-aligned grids, and that patch-agnostic coarse grids really put
triangles across class boundaries (what the coarse-mesh study relies on)."""
import numpy as np

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
