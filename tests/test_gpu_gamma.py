"""GPU parity of the texel-resolution pre-pass and the image-weight mix
(Sec. 3.1, Fig. 5a) against the oracle: visible areas and texel steps bit
for bit, the derived texel layout through the full fusion, and the weight
mix for every rule."""
import numpy as np
import pytest
import torch

import scenegen as sg
from gpu_common import assert_acc_close, check_against_oracle, run_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2111_11103_gb300 import labelfuse as lf
    lf.lib()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def tiny(dev):
    scene, cams = sg.tiny_room(), sg.circle_poses()
    return scene, cams, sg.predictions(scene, cams, "tiny", device=dev)


@pytest.fixture(scope="module")
def medium(dev):
    scene = sg.paper_room(target_faces=60_000)
    cams = sg.random_walk_poses(24, H=151, W=203, fx=183.0, fy=183.0, cx=101.0, cy=75.0)
    return scene, cams, sg.predictions(scene, cams, "paper", device=dev)


def gpu_texel_res(scene, cams, gamma, dev, c):
    from paper_2111_11103_gb300 import labelfuse as lf
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    F = len(scene.faces)
    m = lf.sm_mesh_upload(V, Fc, None, c, "sum", "pixel")
    try:
        s = torch.full((F,), -5, dtype=torch.int32, device=dev)
        a = torch.full((F,), -5, dtype=torch.int32, device=dev)
        lf.sm_texel_res_from_gamma(m, K, T, cams.K.shape[0], cams.H, cams.W, gamma, s, a)
        acc = torch.empty((F, c), device=dev)
        lf.sm_read_state(m, acc, None)
        lf.sm_check(m)
        assert float(acc.abs().max()) == 0.0  # the pre-pass leaves the accumulators alone
    finally:
        lf.sm_mesh_free(m)
    return a.cpu().numpy(), s.cpu().numpy()


@pytest.mark.parametrize("which", ["tiny", "medium"])
@pytest.mark.parametrize("gamma", [0.0, 0.3, 1.0])
def test_areas_and_texel_steps_bit_exact(ora, dev, tiny, medium, which, gamma):
    scene, cams, _ = tiny if which == "tiny" else medium
    a, s = gpu_texel_res(scene, cams, gamma, dev, scene.n_classes)
    a_ora = ora.visible_area(scene.vertices, scene.faces, cams.K, cams.cam_to_world, cams.H, cams.W, nthreads=8)
    assert np.array_equal(a, a_ora)
    assert np.array_equal(s, ora.texel_res_from_gamma(a_ora, gamma))
    assert a.max() > 0


def test_texels_from_gamma_through_fusion(ora, dev, medium):
    """The steps the pre-pass derives define a texel layout that fuses bit for
    bit like the oracle's with the same steps."""
    scene, cams, probs = medium
    _, s = gpu_texel_res(scene, cams, 0.3, dev, scene.n_classes)
    assert s.max() > 1
    res = run_gpu(scene, cams, probs, "logsum", "pixel", texel_res=s, reraster=False)
    check_against_oracle(ora, scene, cams, probs.cpu().numpy(), res, "logsum", "pixel", texel_res=s, nthreads=8)


@pytest.mark.parametrize("rule", ["sum", "logsum", "maxsum", "vote"])
def test_weight_mix_parity(ora, tiny, rule):
    scene, cams, probs = tiny
    res = run_gpu(scene, cams, probs, rule, "image", reraster=False, alpha=0.3)
    check_against_oracle(ora, scene, cams, probs.cpu().numpy(), res, rule, "image", alpha=0.3)


def test_weight_mix_medium_and_endpoints(ora, medium):
    scene, cams, probs = medium
    res = run_gpu(scene, cams, probs, "logsum", "image", reraster=False, alpha=0.6)
    check_against_oracle(ora, scene, cams, probs.cpu().numpy(), res, "logsum", "image", nthreads=8, alpha=0.6)
    # alpha = 0 weighs every pixel 1 (as w^(P)); alpha = 1 is the default w^(I)
    r0 = run_gpu(scene, cams, probs, "sum", "image", reraster=False, alpha=0.0)
    rp = run_gpu(scene, cams, probs, "sum", "pixel", reraster=False)
    assert np.array_equal(r0.cnt, rp.cnt)
    assert_acc_close(r0.acc, rp.acc.astype(np.float64))
    r1 = run_gpu(scene, cams, probs, "sum", "image", reraster=False, alpha=1.0)
    ri = run_gpu(scene, cams, probs, "sum", "image", reraster=False)
    assert_acc_close(r1.acc, ri.acc.astype(np.float64))


def test_f4_invalid_arguments(dev, tiny):
    from paper_2111_11103_gb300 import labelfuse as lf
    scene, cams, _ = tiny
    V, Fc, K, T, _ = to_dev(scene, cams, None, dev)
    F = len(scene.faces)
    s = torch.empty(F, dtype=torch.int32, device=dev)
    mp = lf.sm_mesh_upload(V, Fc, None, 4, "sum", "pixel")
    mi = lf.sm_mesh_upload(V, Fc, None, 4, "sum", "image")
    mt = lf.sm_mesh_upload(V, Fc, torch.full((F,), 2, dtype=torch.int32, device=dev), 4, "sum", "pixel")
    try:
        for call, status in [(lambda: lf.sm_set_weight_mix(mp, 0.5), 1), (lambda: lf.sm_set_weight_mix(mi, 1.5), 1),
                             (lambda: lf.sm_set_weight_mix(mi, float("nan")), 1),
                             (lambda: lf.sm_texel_res_from_gamma(mp, K, T, 8, cams.H, cams.W, -1.0, s), 1),
                             (lambda: lf.sm_texel_res_from_gamma(mp, K, T, 8, cams.H, cams.W, 100.0, s), 1),
                             (lambda: lf.sm_texel_res_from_gamma(mp, K, T, 8, cams.H, cams.W, 0.5, None), 1),
                             (lambda: lf.sm_texel_res_from_gamma(mt, K, T, 8, cams.H, cams.W, 0.5, s), 4)]:
            with pytest.raises(lf.LabelFuseError) as e:
                call()
            assert e.value.status == status
        lf.sm_set_weight_mix(mi, 0.0)
        lf.sm_texel_res_from_gamma(mp, K, T, 0, cams.H, cams.W, 0.5, s)  # no frames: s = 1
        assert int(s.min()) == 1 and int(s.max()) == 1
    finally:
        for m in (mp, mi, mt):
            lf.sm_mesh_free(m)
