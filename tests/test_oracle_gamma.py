"""Pins for the texel-resolution pre-pass and the weight mix (Sec. 3.1 and
Fig. 5a): hand-worked s_t values, hand-counted visible areas (maximum over
frames, not a sum), brute-force areas from the row maps, an independent
binary32 evaluation, and the weight mix's endpoints, linearity in alpha and
mass conservation."""
import os

import numpy as np
import pytest

import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
IDENT = np.eye(4)


def _cases():
    rows = []
    for line in open(os.path.join(GOLDEN, "texel_steps_gamma.txt")):
        line = line.split("#")[0].strip()
        if line:
            name, a, g, s = line.split()
            rows.append((name, int(a), float(g), int(s)))
    return rows


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_texel_steps_hand_values(ora, case):
    name, a, g, s = case
    assert ora.texel_res_from_gamma(np.array([a]), g)[0] == s


def test_texel_steps_binary32(ora):
    """The decision is taken in binary32; numpy's float32 sqrt / multiply /
    ceil (an independent IEEE implementation) agree on random inputs."""
    rng = np.random.default_rng(5)
    a = rng.integers(0, 400_000, size=20_000)
    for g in (0.05, 0.1, 0.37, 1.0, 2.5):
        ref = np.maximum(1, np.ceil(np.float32(g) * np.sqrt(a.astype(np.float32))).astype(np.int64))
        assert np.array_equal(ora.texel_res_from_gamma(a, g), ref)


def test_visible_area_hand_counted(ora):
    """The integer right triangle covers 36 pixel centres (hand count); seen in
    two identical frames and one where it is off screen, a_t stays 36 (the
    maximum over frames, not their sum)."""
    V = np.array([[0, 0, 1], [8, 0, 1], [0, 8, 1]], dtype=np.float32)
    K = np.array([[1.0, 1.0, 0.0, 0.0], [1.0, 1.0, 0.0, 0.0], [1.0, 1.0, 100.0, 0.0]])
    T = np.stack([IDENT] * 3)
    assert list(ora.visible_area(V, [[0, 1, 2]], K, T, 16, 16)) == [36]
    assert list(ora.visible_area(V, [[0, 1, 2]], K[2:], T[2:], 16, 16)) == [0]


def test_visible_area_is_max_of_per_frame_counts(ora):
    scene, cams = sg.tiny_room(), sg.circle_poses()
    mesh = ora.Mesh(scene.vertices, scene.faces)
    per_frame = [np.bincount(ora.render_frame(mesh, cams.K[i], cams.cam_to_world[i], cams.H, cams.W).ravel() + 1,
                             minlength=len(scene.faces) + 1)[1:] for i in range(cams.K.shape[0])]
    expect = np.max(per_frame, axis=0)
    for nt in (1, 3):
        got = ora.visible_area(scene.vertices, scene.faces, cams.K, cams.cam_to_world, cams.H, cams.W, nthreads=nt)
        assert np.array_equal(got, expect)
    assert expect.max() > 0


@pytest.fixture(scope="module")
def tiny_fused(ora):
    scene, cams = sg.tiny_room(), sg.circle_poses()
    probs = sg.predictions(scene, cams, "tiny", device="cpu").numpy()
    mesh = ora.Mesh(scene.vertices, scene.faces)
    return scene, cams, probs, mesh


@pytest.mark.parametrize("rule", ["sum", "logsum"])
def test_weight_mix_endpoints_and_linearity(ora, tiny_fused, rule):
    scene, cams, probs, mesh = tiny_fused
    run = lambda w, a: ora.fuse_sequence(mesh, cams.K, cams.cam_to_world, probs, rule, w, alpha=a)[0]
    A_pix, A_img = run("pixel", 1.0), run("image", 1.0)
    assert np.array_equal(run("image", 0.0), A_pix)  # (1 - 0) + 0 / n = 1 exactly
    for a in (0.25, 0.7):
        np.testing.assert_allclose(run("image", a), (1 - a) * A_pix + a * A_img, rtol=1e-12, atol=1e-12)


def test_weight_mix_mass(ora, tiny_fused):
    """sum rule: each row's mass is sum_i n_i ((1 - a) + a / n_i) =
    (1 - a) cnt + a (number of frames that see the row)."""
    scene, cams, probs, mesh = tiny_fused
    a = 0.4
    A, cnt = ora.fuse_sequence(mesh, cams.K, cams.cam_to_world, probs, "sum", "image", alpha=a)
    frames = np.zeros(mesh.n_x)
    for i in range(cams.K.shape[0]):
        idm = ora.render_frame(mesh, cams.K[i], cams.cam_to_world[i], cams.H, cams.W)
        frames[np.unique(idm[idm >= 0])] += 1
    np.testing.assert_allclose(A.sum(1), (1 - a) * cnt + a * frames, rtol=1e-6)
