"""Planted mistakes in a copy of the oracle make its pins fail.

Each case copies ``oracle/``, ``scenegen/`` and the oracle's pin tests into a
temporary tree, plants ONE plausible mistake in the copy (a flipped fill rule,
a dropped term, a transposed operand, a wrong sign or index ...), and runs the
pins there in a subprocess: pytest must report failing tests (exit status 1,
not a crash and not a pass).  The repository's oracle is never modified.  The
mutants run concurrently, once per session.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["test_oracle_raster.py", "test_oracle_texels.py", "test_oracle_fusion.py", "test_oracle_gamma.py",
             "test_oracle_confidence.py"]

C, PY = "oracle/oracle.c", "oracle/confidence.py"

# name -> (file, original text, planted mistake)
MUTANTS = {
    # renderer (Sec. 3.3.1)
    "fill_rule_bottom_right": (C, "return dy < 0 || (dy == 0 && dx > 0);", "return dy > 0 || (dy == 0 && dx < 0);"),
    "edges_all_exclusive": (C, "if (E[k] == 0 && !ora_top_left(t, k)) return 0;", "if (E[k] == 0) return 0;"),
    "edge_operands_transposed": (C, "return dx * (py - t->y[b]) - dy * (px - t->x[b]);",
                                 "return dx * (px - t->x[b]) - dy * (py - t->y[b]);"),
    "depth_term_dropped": (C, "float num = (w[0] + w[1]) + w[2];", "float num = w[0] + w[1];"),
    "farthest_surface_wins": (C, "uint64_t key = ((uint64_t)(0xFFFFFFFFu - ora_float_bits(inv_z)) << 32)",
                              "uint64_t key = ((uint64_t)ora_float_bits(inv_z) << 32)"),
    "near_plane_at_zero": (C, "if (!(Z > ORA_Z_NEAR)) return 0;", "if (!(Z > 0.0f)) return 0;"),
    "last_column_clipped": (C, "if (x1 > W - 1) x1 = W - 1;", "if (x1 > W - 2) x1 = W - 2;"),
    "pose_not_inverted": (C, "for (int c = 0; c < 3; ++c) R[r][c] = T[c * 4 + r];",
                          "for (int c = 0; c < 3; ++c) R[r][c] = T[r * 4 + c];"),
    "camera_centre_sign": (C, "for (int r = 0; r < 3; ++r) t[r] = -((R[r][0] * C[0]",
                           "for (int r = 0; r < 3; ++r) t[r] = ((R[r][0] * C[0]"),
    "principal_point_dropped": (C, "A[c] = (float)(256.0 * (fx * R[0][c] + cx * R[2][c]));",
                                "A[c] = (float)(256.0 * (fx * R[0][c]));"),
    # texels (Sec. 3.1)
    "texel_count_off_by_one": (C, "int64_t ora_texel_count(int64_t s) { return (s * s + s) / 2; }",
                               "int64_t ora_texel_count(int64_t s) { return (s * s - s) / 2; }"),
    "texel_id_triangular_off_by_one": (C, "return n * (n + 1) / 2 + j;", "return n * (n - 1) / 2 + j;"),
    "texel_cell_clamp_to_square": (C, "if (j > s - 1 - i) j = s - 1 - i;", "if (j > s - 1) j = s - 1;"),
    "uv_axes_swapped": (C, "float u = beta[(o + 1) % 3], v = beta[(o + 2) % 3];",
                        "float u = beta[(o + 2) % 3], v = beta[(o + 1) % 3];"),
    "uv_origin_farthest_from_right_angle": (C, "if (k == 0 || q < best) {", "if (k == 0 || q > best) {"),
    "barycentrics_ignore_orientation_fix": (C, "for (int k = 0; k < 3; ++k) beta[t.local[k]] = w[k] / num;",
                                            "for (int k = 0; k < 3; ++k) beta[k] = w[k] / num;"),
    "row_offsets_inclusive": (C, "        id_t[f] = acc;\n        acc += ora_texel_count(s ? (int64_t)s[f] : 1);",
                              "        acc += ora_texel_count(s ? (int64_t)s[f] : 1);\n        id_t[f] = acc;"),
    # aggregation (Sec. 3.2)
    "image_weight_ignored": (C, "w_out[k] = (1.0 - alpha) + alpha / (double)counts[idmap[k]];", "w_out[k] = 1.0;"),
    "weight_mix_reversed": (C, "w_out[k] = (1.0 - alpha) + alpha / (double)counts[idmap[k]];",
                            "w_out[k] = alpha + (1.0 - alpha) / (double)counts[idmap[k]];"),
    "weight_not_applied": (C, "A[(int64_t)l * c + j] += w * phi[j];", "A[(int64_t)l * c + j] += phi[j];"),
    "count_doubled": (C, "        cnt[l] += 1;\n    }\n    free(phi);", "        cnt[l] += 2;\n    }\n    free(phi);"),
    "maxsum_keeps_one": (C, "case ORA_RULE_MAXSUM: out[j] = (p[j] == m) ? (double)p[j] : 0.0; break;",
                         "case ORA_RULE_MAXSUM: out[j] = (p[j] == m) ? 1.0 : 0.0; break;"),
    "maxsum_keeps_all": (C, "case ORA_RULE_MAXSUM: out[j] = (p[j] == m) ? (double)p[j] : 0.0; break;",
                         "case ORA_RULE_MAXSUM: out[j] = (double)p[j]; break;"),
    "logsum_base_10": (C, "out[j] = log(q > ORA_P_MIN ? q : ORA_P_MIN);", "out[j] = log10(q > ORA_P_MIN ? q : ORA_P_MIN);"),
    "logsum_without_clamp": (C, "out[j] = log(q > ORA_P_MIN ? q : ORA_P_MIN);", "out[j] = log(q);"),
    "vote_is_sum": (C, "default: out[j] = (j == am) ? 1.0 : 0.0; break;", "default: out[j] = (double)p[j]; break;"),
    "argmax_ties_to_last": (C, "            if (a[j] > a[am]) am = j;", "            if (a[j] >= a[am]) am = j;"),
    "logsum_normalised_as_sum": (C, "if (rule == ORA_RULE_LOGSUM) {\n            for (int32_t j = 0; j < c; ++j) total += exp",
                                 "if (rule == -1) {\n            for (int32_t j = 0; j < c; ++j) total += exp"),
    "unseen_rows_labelled_zero": (C, "if (labels) labels[l] = -1;", "if (labels) labels[l] = 0;"),
    "background_rendered_zero": (C, "out[k] = (l < 0 || labels[l] < 0) ? (uint8_t)255 : (uint8_t)labels[l];",
                                 "out[k] = (l < 0 || labels[l] < 0) ? (uint8_t)0 : (uint8_t)labels[l];"),
    # texel resolution from gamma (Sec. 3.1)
    "gamma_steps_floor": (C, "const float c = ceilf(g);", "const float c = floorf(g);"),
    "visible_area_summed": (C, "if (count[f] > j->area[f]) j->area[f] = count[f];", "j->area[f] += count[f];"),
    "snap_by_floor": (C, "*xs = (int64_t)rintf(xf);", "*xs = (int64_t)floorf(xf);"),
    "depth_not_divided_by_area": (C, "return num / (float)t->area2;", "return num;"),
    # whole sequences on several threads
    "thread_partials_overwritten": (C, "for (int64_t q = 0; q < n_x * c; ++q) A[q] += jobs[t].A[q];",
                                    "for (int64_t q = 0; q < n_x * c; ++q) A[q] = jobs[t].A[q];"),
    "thread_counts_dropped": (C, "for (int64_t l = 0; l < n_x; ++l) cnt[l] += jobs[t].cnt[l];", ""),
    "area_thread_maxima_dropped": (C, "if (jobs[t].area[f] > area_out[f]) area_out[f] = jobs[t].area[f];", ";"),
    "render_sequence_one_frame_slot": (C, "j->T + 16 * (int64_t)i, j->H, j->W, j->idmaps_out + (int64_t)i * npix, NULL, NULL) < 0)",
                                       "j->T + 16 * (int64_t)i, j->H, j->W, j->idmaps_out, NULL, NULL) < 0)"),
    # learned confidence
    "conf_sigmoid_sign": (PY, "q = 1.0 / (1.0 + np.exp(-o))", "q = 1.0 / (1.0 + np.exp(o))"),
    "conf_weight_unclipped": (PY, "w = np.maximum(o, W_FLOOR)", "w = np.abs(o)"),
    "conf_weight_is_probability": (PY, "w = np.maximum(o, W_FLOOR)", "w = 1.0 / (1.0 + np.exp(-o))"),
    "conf_weight_floor_zero": (PY, "w = np.maximum(o, W_FLOOR)", "w = np.maximum(o, 0.0)"),
    "conf_loss_sign": (PY, "loss = np.mean(np.logaddexp(0.0, o) - y * o)", "loss = np.mean(np.logaddexp(0.0, o) + y * o)"),
    "conf_depth_scale": (PY, "1.0 / np.where(invz > 0, invz, 1.0), 0.0) / 4.0", "1.0 / np.where(invz > 0, invz, 1.0), 0.0) / 2.0"),
    "conf_cos_not_absolute": (PY, "cos = np.abs((n * ray).sum(1))", "cos = ((n * ray).sum(1))"),
    "conf_backward_transposed": (PY, "d_z1 = (d_z2 @ W2) * (z1 > 0)", "d_z1 = (d_z2 @ W2.T) * (z1 > 0)"),
    "conf_relu_dropped": (PY, "h2 = np.maximum(z2, 0.0)", "h2 = z2"),
    "conf_bias_gradient_dropped": (PY, "g_b1 = d_z1.sum(0)", "g_b1 = 0.0 * d_z1.sum(0)"),
    "conf_entropy_unnormalised": (PY, ".sum(1) / np.log(c) if c > 1", ".sum(1) if c > 1"),
    "conf_border_off_by_one": (PY, "np.minimum(W - 1 - xs, H - 1 - ys)", "np.minimum(W - xs, H - ys)"),
    "conf_target_compares_row_id": (PY, "return ((rows >= 0) & (am == lab)).astype(np.float64)",
                                    "return ((rows >= 0) & (am == rows)).astype(np.float64)"),
    "conf_bf16_ties_away": (PY, "rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000",
                            "rounded = (u + 0x8000) & 0xFFFF0000"),
}


def _run_mutant(name: str, spec, base: str):
    path, old, new = spec
    tree = os.path.join(base, name)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tree, "oracle"),
                    ignore=shutil.ignore_patterns("*.so", "*.so.*", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "scenegen"), os.path.join(tree, "scenegen"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(tree, "tests"))
    for f in PIN_FILES + ["conftest.py"]:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(tree, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tree, "tests", "golden"))
    target = os.path.join(tree, path)
    src = open(target).read()
    if src.count(old) != 1:
        return name, None, f"planting site not found exactly once: {old!r}"
    with open(target, "w") as fh:
        fh.write(src.replace(old, new, 1))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_FILES],
                       cwd=os.path.join(tree, "tests"), capture_output=True, text=True, env=env, timeout=600)
    return name, r.returncode, (r.stdout + r.stderr)[-600:]


@pytest.fixture(scope="module")
def mutant_results():
    base = tempfile.mkdtemp(prefix="oracle_mutants_")
    try:
        workers = max(1, min(8, os.cpu_count() or 1))
        with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
            out = list(ex.map(lambda n: _run_mutant(n, MUTANTS[n], base), sorted(MUTANTS)))
        return {name: (rc, tail) for name, rc, tail in out}
    finally:
        shutil.rmtree(base, ignore_errors=True)


def test_unmodified_copy_passes():
    """The copying itself leaves the pins green (no false kills)."""
    base = tempfile.mkdtemp(prefix="oracle_copy_")
    try:
        same = "int64_t ora_texel_count(int64_t s)"
        _, rc, tail = _run_mutant("identity", (C, same, same), base)
        assert rc == 0, tail
    finally:
        shutil.rmtree(base, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(mutant_results, name):
    rc, tail = mutant_results[name]
    assert rc == 1, f"{name}: pins exit status {rc} (1 = a pin failed)\n{tail}"
