"""Host helpers of the benchmark: the storage-form quantiser (per-pixel scale,
BF16 / E4M3 codes) and the lookup of the committed scatter profile."""
import importlib.util
import os

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_quantise_scales_and_codes():
    b = _bench()
    g = torch.Generator().manual_seed(0)
    probs = torch.softmax(torch.randn((3, 5, 7, 40), generator=g), -1)
    for kind, top in (("bf16", 1.0), ("fp8_e4m3", 448.0)):
        q, scale = b.quantise(probs, kind)
        assert q.shape == probs.shape and scale.shape == probs.shape[:-1]
        np.testing.assert_allclose(scale.numpy(), probs.amax(-1).numpy() / top, rtol=1e-7)
        deq = (q.float() * scale[..., None]).numpy()
        p, s = probs.numpy(), scale[..., None].numpy()
        if kind == "bf16":  # 8 significant bits: half an ulp is 2^-8 relative
            bound = 2.0 ** -8 * p + 1e-12
        else:  # E4M3: 4 significant bits (2^-4 relative), subnormal step 2^-9 of the scale
            bound = 2.0 ** -4 * p + 2.0 ** -10 * s + 1e-12
        assert np.all(np.abs(deq - p) <= bound)
        assert float(q.float().amax()) == top  # the largest class maps to the top code exactly


def test_traffic_lookup_follows_the_source_hash(tmp_path, monkeypatch):
    """The committed capture's traffic is used only while the kernel sources
    it was taken on are unchanged; then it is a plausible per-frame figure."""
    b = _bench()
    for kern in ("scatter", "queue"):
        tpf = b.kernel_traffic_per_frame(kern)
        assert tpf is None or (5.0e7 < tpf[0] < 7.0e7 and tpf[1] >= 1)  # bytes per 640 x 480 x 40 frame
    assert b.kernel_traffic_per_frame("render") is None
    # a summary whose hash matches is read; any other hash is ignored
    sha = b.source_sha(b.TRAFFIC["scatter"][1])
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "scatter_paper_room.md").write_text(
        f"x\n    traffic_bytes_per_launch: 4400000000\n    frames_per_launch: 84\n    source_sha: {sha}\n")
    csrc = os.path.join(ROOT, "paper_2111_11103_gb300", "csrc")
    (tmp_path / "paper_2111_11103_gb300").mkdir()
    os.symlink(csrc, tmp_path / "paper_2111_11103_gb300" / "csrc")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.kernel_traffic_per_frame("scatter") == (4400000000 / 84, 84)
    (prof / "scatter_paper_room.md").write_text(
        "x\n    traffic_bytes_per_launch: 4400000000\n    frames_per_launch: 84\n    source_sha: 0000000000000000\n")
    assert b.kernel_traffic_per_frame("scatter") is None


def test_l2_note_states_the_resident_size():
    import bench
    assert bench.l2_note(49_152_000_000).startswith("inputs larger than L2 (49.2 GB")
    assert "NOT larger than L2" in bench.l2_note(100 << 20)


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` (the oracle timed on the host cores) runs on
    a machine without a GPU and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--faces", "20000", "--frames", "16", "--cpu-frames", "4"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cfg = d["config"]
    assert (cfg["H"], cfg["W"], cfg["classes"], cfg["frames"]) == (480, 640, 40, 16)
    assert abs(cfg["faces"] - 20000) <= 200 and cfg["rule"] == "logsum" and cfg["weight"] == "pixel"


def test_gpus_flag_launches_that_many_ranks():
    """`bench.py --gpus 2` outside a launcher re-runs itself as two ranks under
    torchrun (rendezvous on 127.0.0.1); in --dry-run mode the ranks join a
    gloo group and rank 0 prints every rank's share of the frames."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--dry-run", "--frames", "1000"],
                       cwd=root, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["n_ranks"] == 2 and d["processes"] == 2
    assert d["frame_ranges"] == [[0, 500], [500, 1000]]


def test_gpus_flag_must_match_the_launcher():
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WORLD_SIZE="4", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--dry-run"], cwd=root, capture_output=True,
                       text=True, timeout=600, env=env)
    assert r.returncode != 0 and "WORLD_SIZE=4" in r.stderr


def test_kernel_times_on_the_step_stream_stay_within_the_step():
    """The per-kernel breakdown holds only the kernels on the step's stream;
    the raster's event span (second stream, waits included) is reported apart."""
    prof = {"project": (1, 0.2), "raster": (4, 160.0), "scatter": (2, 190.0), "normalise": (1, 0.4),
            "render": (1, 5.6), "resolve": (0, 0.0)}
    bench = _bench()
    kernels, raster = bench.split_kernel_times(prof, 20)
    assert set(kernels) == {"project", "scatter", "normalise", "render"}
    assert abs(sum(v["ms_per_step"] for v in kernels.values()) - (0.2 + 190.0 + 0.4 + 5.6) / 20) < 1e-12
    assert raster["launches"] == 4 and raster["event_span_ms_per_step"] == 8.0 and "span" in raster["note"]
    assert bench.split_kernel_times({"scatter": (1, 1.0)}, 1)[1] is None
