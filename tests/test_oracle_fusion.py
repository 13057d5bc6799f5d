"""Pins for the oracle's aggregation (Sec. 3.2): fusion rules f_sum, f_mul,
f_maxsum (Eqs. sum, mul, maxsum), their weighted forms with w^(P) and w^(I)
(Sec. 3.2.2), normalisation and arg max (Sec. 3.2.1), render-back, and the
permutation invariance the paper states (Sec. 3.3.2)."""
import numpy as np
import pytest


def _softmax(x):
    e = np.exp(x - x.max(-1, keepdims=True))
    return (e / e.sum(-1, keepdims=True)).astype(np.float32)


def test_one_pixel_one_frame(ora):
    """f_sum and f_mul of a single observation reproduce it (normalised)."""
    rng = np.random.default_rng(0)
    p = _softmax(rng.normal(size=(1, 7)))
    ref = p[0].astype(np.float64) / p[0].astype(np.float64).sum()
    for rule in ("sum", "logsum"):
        A, cnt = ora.accumulate(rule, [0], p, n_x=1)
        d, lab = ora.normalise(rule, A, cnt)
        np.testing.assert_allclose(d[0], ref, rtol=1e-14, atol=0)
        assert lab[0] == int(np.argmax(p[0]))


def test_constant_prediction_closed_forms(ora):
    """All n pixels of a row carry the same p.  w^(I), one frame: sum and mul
    give norm(p).  w^(P): sum gives norm(p), mul gives norm(p^n)."""
    rng = np.random.default_rng(1)
    p = _softmax(rng.normal(size=(1, 5)))[0]
    n = 9
    idmap = np.zeros((1, 3, 3), dtype=np.int32)
    probs = np.broadcast_to(p, (1, 3, 3, 5)).copy()
    p64 = p.astype(np.float64)
    for weight in ("image", "pixel"):
        for rule in ("sum", "logsum"):
            A, cnt = ora.fuse_frames(rule, weight, idmap, probs, n_x=1)
            d, _ = ora.normalise(rule, A, cnt)
            if rule == "logsum" and weight == "pixel":
                expect = p64 ** n / (p64 ** n).sum()
            else:
                expect = p64 / p64.sum()
            np.testing.assert_allclose(d[0], expect, rtol=1e-12)
            assert cnt[0] == n


def test_mul_equals_direct_product(ora):
    """The log-domain f_w-mul equals norm(prod p^w) computed directly (no underflow)."""
    rng = np.random.default_rng(2)
    probs = _softmax(rng.normal(size=(2, 4, 4, 6)))
    idmaps = rng.integers(0, 3, size=(2, 4, 4)).astype(np.int32)
    for weight in ("pixel", "image"):
        A, cnt = ora.fuse_frames("logsum", weight, idmaps, probs, n_x=3)
        d, lab = ora.normalise("logsum", A, cnt)
        for l in range(3):
            prod = np.ones(6)
            for i in range(2):
                m = idmaps[i] == l
                w = 1.0 / m.sum() if weight == "image" and m.sum() else 1.0
                for pk in probs[i][m]:
                    prod *= pk.astype(np.float64) ** w
            np.testing.assert_allclose(d[l], prod / prod.sum(), rtol=1e-10)
            assert lab[l] == int(np.argmax(prod))


def test_maxsum_g_function(ora):
    """g keeps every entry equal to max p (ties included) and zeroes the rest."""
    p = np.array([0.1, 0.4, 0.1, 0.4], dtype=np.float32)
    np.testing.assert_array_equal(ora.phi("maxsum", p), [0, np.float32(0.4), 0, np.float32(0.4)])
    q = np.array([0.7, 0.1, 0.2], dtype=np.float32)
    np.testing.assert_array_equal(ora.phi("maxsum", q), [np.float32(0.7), 0, 0])
    # vote: one-hot at the first arg max
    np.testing.assert_array_equal(ora.phi("vote", p), [0, 1, 0, 0])
    np.testing.assert_array_equal(ora.phi("sum", q), q.astype(np.float64))
    lg = ora.phi("logsum", np.array([0.5, 0.0], dtype=np.float32))
    assert lg[0] == np.log(np.float64(np.float32(0.5))) and lg[1] == np.log(2.0 ** -30)


def test_maxsum_hand_example(ora):
    """Two pixels of one row: f_maxsum = norm(g(p1) + g(p2))."""
    p = np.array([[0.5, 0.3, 0.2], [0.25, 0.45, 0.3]], dtype=np.float32)
    A, cnt = ora.accumulate("maxsum", [0, 0], p, n_x=1)
    np.testing.assert_allclose(A[0], [np.float32(0.5), np.float32(0.45), 0.0], rtol=0)
    d, lab = ora.normalise("maxsum", A, cnt)
    np.testing.assert_allclose(d[0], np.array([0.5, 0.45, 0.0]) / 0.95, rtol=1e-7)
    assert lab[0] == 0


@pytest.mark.parametrize("rule", ["sum", "logsum", "maxsum", "vote"])
def test_image_weights(ora, rule):
    """w^(I) = 1/|K_i ∩ K_x|: each frame adds total weight 1 to each row it sees."""
    rng = np.random.default_rng(3)
    N, H, W, c, n_x = 5, 6, 7, 4, 9
    probs = _softmax(rng.normal(size=(N, H, W, c)))
    idmaps = rng.integers(-1, n_x, size=(N, H, W)).astype(np.int32)
    A, cnt = ora.fuse_frames(rule, "image", idmaps, probs, n_x=n_x)
    frames_seeing = np.array([sum(np.any(idmaps[i] == l) for i in range(N)) for l in range(n_x)])
    if rule in ("sum", "vote"):
        np.testing.assert_allclose(A.sum(1), frames_seeing, rtol=1e-6)
    w = ora.frame_weights("image", idmaps[0], n_x)
    for l in range(n_x):
        m = idmaps[0].ravel() == l
        if m.any():
            assert np.allclose(w[m], 1.0 / m.sum())
    assert np.all(w[idmaps[0].ravel() < 0] == 0)


def test_mass_and_coverage_conservation(ora):
    """w^(P): sum_j A_sum[l][j] = pixels on l (probabilities sum to 1 up to
    binary32 rounding); sum_l cnt[l] = covered pixels."""
    rng = np.random.default_rng(4)
    N, H, W, c, n_x = 4, 8, 9, 6, 11
    probs = _softmax(rng.normal(size=(N, H, W, c)))
    idmaps = rng.integers(-1, n_x, size=(N, H, W)).astype(np.int32)
    A, cnt = ora.fuse_frames("sum", "pixel", idmaps, probs, n_x=n_x)
    np.testing.assert_allclose(A.sum(1), cnt, rtol=1e-6)
    assert cnt.sum() == (idmaps >= 0).sum()
    for l in range(n_x):
        assert cnt[l] == (idmaps == l).sum()


@pytest.mark.parametrize("rule", ["sum", "logsum", "maxsum", "vote"])
@pytest.mark.parametrize("weight", ["pixel", "image"])
def test_frame_order_invariance(ora, rule, weight):
    """Aggregation is permutation invariant (Sec. 3.3.2): a random frame order
    agrees to 1e-12 relative in binary64."""
    rng = np.random.default_rng(5)
    N, H, W, c, n_x = 12, 5, 6, 5, 7
    probs = _softmax(rng.normal(size=(N, H, W, c)))
    idmaps = rng.integers(-1, n_x, size=(N, H, W)).astype(np.int32)
    A1, c1 = ora.fuse_frames(rule, weight, idmaps, probs, n_x=n_x)
    perm = rng.permutation(N)
    A2, c2 = ora.fuse_frames(rule, weight, idmaps[perm], probs[perm], n_x=n_x)
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_allclose(A1, A2, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("rule", ["sum", "logsum"])
def test_frame_shard_associativity(ora, rule):
    """Fusing disjoint frame shards and adding the accumulators equals fusing
    all frames (every rule is a sum, Sec. 3.3.2)."""
    rng = np.random.default_rng(6)
    N, H, W, c, n_x = 9, 5, 5, 3, 6
    probs = _softmax(rng.normal(size=(N, H, W, c)))
    idmaps = rng.integers(-1, n_x, size=(N, H, W)).astype(np.int32)
    A, cnt = ora.fuse_frames(rule, "image", idmaps, probs, n_x=n_x)
    As, cs = np.zeros_like(A), np.zeros_like(cnt)
    for r in range(3):
        a, k = ora.fuse_frames(rule, "image", idmaps[r::3], probs[r::3], n_x=n_x)
        As += a
        cs += k
    np.testing.assert_array_equal(cs, cnt)
    np.testing.assert_allclose(As, A, rtol=1e-12)


def test_unseen_rows_and_render_back(ora):
    """Rows never observed stay unlabelled (-1, zero distribution) and render as
    255, like background pixels."""
    probs = _softmax(np.array([[[[2.0, 0.0, 1.0]]]]))
    idmaps = np.array([[[1]]], dtype=np.int32)
    A, cnt = ora.fuse_frames("sum", "pixel", idmaps, probs, n_x=3)
    d, lab = ora.normalise("sum", A, cnt)
    assert list(lab) == [-1, 0, -1]
    assert np.all(d[0] == 0) and np.all(d[2] == 0)
    out = ora.render_labels(np.array([[0, 1, 2, -1]], dtype=np.int32), lab)
    assert out.tolist() == [[255, 0, 255, 255]]


def test_normalised_rows_sum_to_one(ora):
    rng = np.random.default_rng(7)
    probs = _softmax(3 * rng.normal(size=(3, 6, 6, 10)))
    idmaps = rng.integers(0, 4, size=(3, 6, 6)).astype(np.int32)
    for rule in ("sum", "logsum", "maxsum", "vote"):
        A, cnt = ora.fuse_frames(rule, "pixel", idmaps, probs, n_x=4)
        d, lab = ora.normalise(rule, A, cnt)
        np.testing.assert_allclose(d.sum(1), 1.0, rtol=0, atol=1e-15)
        assert np.array_equal(lab, np.argmax(A, 1))


def test_argmax_ties_lowest_index(ora):
    A = np.array([[1.0, 3.0, 3.0, 0.0]])
    _, lab = ora.normalise("sum", A, np.array([2]))
    assert lab[0] == 1


def test_sequence_matches_framewise(ora):
    """The threaded whole-sequence driver equals frame-by-frame rendering and
    fusion, for any thread count (tiny room, 8 frames)."""
    import scenegen as sg
    sc = sg.tiny_room()
    cams = sg.circle_poses()
    probs = sg.predictions(sc, cams, "tiny").numpy()
    mesh = ora.Mesh(sc.vertices, sc.faces)
    idm = np.stack([ora.render_frame(mesh, cams.K[i], cams.cam_to_world[i], cams.H, cams.W) for i in range(8)])
    A0, c0 = ora.fuse_frames("logsum", "image", idm, probs, mesh.n_x)
    for nt in (1, 3):
        A1, c1, idm1 = ora.fuse_sequence(mesh, cams.K, cams.cam_to_world, probs, "logsum", "image", nthreads=nt,
                                         want_idmaps=True)
        assert np.array_equal(idm1, idm)
        np.testing.assert_array_equal(c1, c0)
        np.testing.assert_allclose(A1, A0, rtol=1e-12)
    # the plain method improves on the raw predictions on this easy scene
    _, lab = ora.normalise("logsum", A0, c0)
    seen = c0 > 0
    assert np.mean(lab[seen] == sc.face_gt[seen]) > 0.95
