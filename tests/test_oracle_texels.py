"""Pins for the oracle's texel parametrisation (Sec. 3.1, Fig. 3, Eq. idtexel,
Eq. texel-in-array), checked against values the paper prints and against
properties fixed by the mathematics."""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = int(v)
    return out


def test_texel_count_matches_paper(ora):
    g = _golden("paper_worked_examples.txt")
    assert ora.texel_count(6) == g["texel_count_s6"]
    assert ora.texel_count(1) == g["texel_count_s1"]


@pytest.mark.parametrize("s", list(range(1, 65)))
def test_texel_id_is_bijection(ora, s):
    """Every cell (i, j) with i + j < s gets a distinct id in [0, (s^2+s)/2)."""
    ids = sorted(ora.texel_id(i, j) for i in range(s) for j in range(s - i))
    assert ids == list(range(ora.texel_count(s)))


def test_printed_texel_formula_collides():
    """The printed Eq. (idtexel), T(floor(su)) + floor(sv), is not injective on
    the triangle's cells (the reason for the reading used by the oracle)."""
    s = 2
    printed = {(i, j): i * (i + 1) // 2 + j for i in range(s) for j in range(s - i)}
    assert len(set(printed.values())) < len(printed)


def test_texel_cells_cover_triangle(ora):
    """A uv point's cell contains it (up to the clamp at the u + v = 1 edge):
    brute force over a grid of uv points, checked against floor(s*u), floor(s*v)
    computed independently in binary64."""
    rng = np.random.default_rng(0)
    for s in (1, 2, 3, 6, 17):
        for _ in range(400):
            u, v = rng.uniform(0, 1, size=2)
            if u + v >= 1:
                u, v = 1 - u, 1 - v
            u32, v32 = np.float32(u), np.float32(v)
            i, j = ora.texel_cell(s, u32, v32)
            assert 0 <= i and 0 <= j and i + j <= s - 1
            fi, fj = int(np.floor(s * float(u32))), int(np.floor(s * float(v32)))
            if fi + fj <= s - 1 and fi <= s - 1:
                # away from the clamp the cell is exactly the floor pair, unless
                # the binary32 product rounds across an integer
                if abs(s * float(u32) - round(s * float(u32))) > 1e-5 and abs(s * float(v32) - round(s * float(v32))) > 1e-5:
                    assert (i, j) == (fi, fj)


def test_texel_cell_clamps(ora):
    assert ora.texel_cell(4, 1.0, 0.0) == (3, 0)
    assert ora.texel_cell(4, 0.0, 1.0) == (0, 3)
    assert ora.texel_cell(4, 0.5, 0.5) == (2, 1)   # u + v = 1 rounds onto the edge: j clamped
    assert ora.texel_cell(1, 0.7, 0.2) == (0, 0)


def test_uv_origin_right_angle(ora):
    """The origin is the vertex at the interior angle closest to 90 degrees."""
    right = [np.array([0.0, 0.0, 0.0]), np.array([2.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])]
    for perm in itertools.permutations(range(3)):
        pts = [right[k] for k in perm]
        assert ora.uv_origin(*pts) == perm.index(0)
    # obtuse triangle: angles ~ 120, 30, 30 deg -> the 120 deg vertex (|120-90| = 30 < 60)
    obtuse = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([-0.5, np.sqrt(3) / 2, 0.0])]
    assert ora.uv_origin(*obtuse) == 0
    # angles 100, 40, 40 deg -> the 100 deg vertex
    a = np.radians(100.0)
    tri = [np.zeros(3), np.array([1.0, 0.0, 0.0]), np.array([np.cos(a), np.sin(a), 0.0])]
    assert ora.uv_origin(*tri) == 0
    # equilateral: all tie -> lowest local index
    eq = [np.array([0.0, 0.0, 0.0]), np.array([1.0, 0.0, 0.0]), np.array([0.5, np.sqrt(3) / 2, 0.0])]
    assert ora.uv_origin(*eq) == 0


def test_uv_origin_brute_force(ora):
    """Against angles computed with arccos in binary64 on random triangles
    (skipping near-ties)."""
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(2000):
        P = rng.normal(size=(3, 3)).astype(np.float32).astype(np.float64)
        dev = []
        for k in range(3):
            e1, e2 = P[(k + 1) % 3] - P[k], P[(k + 2) % 3] - P[k]
            ang = np.degrees(np.arccos(np.clip(e1 @ e2 / np.linalg.norm(e1) / np.linalg.norm(e2), -1, 1)))
            dev.append(abs(ang - 90.0))
        order = np.argsort(dev)
        if dev[order[1]] - dev[order[0]] < 1e-3:
            continue
        assert ora.uv_origin(P[0], P[1], P[2]) == order[0]
        checked += 1
    assert checked > 1900


def test_row_offsets(ora):
    id_t, n_x = ora.row_offsets(5)
    assert n_x == 5 and list(id_t) == [0, 1, 2, 3, 4, 5]
    s = np.array([1, 6, 2, 1, 3], dtype=np.int32)
    id_t, n_x = ora.row_offsets(5, s)
    assert list(id_t) == [0, 1, 22, 25, 26, 32] and n_x == 32
    id_t, n_x = ora.row_offsets(0)
    assert n_x == 0 and list(id_t) == [0]
