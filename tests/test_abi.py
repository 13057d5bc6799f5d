"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/labelfuse.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "labelfuse.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2111_11103_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sm_mesh_upload", "sm_fuse_frames", "sm_normalise", "sm_render_labels"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2111_11103_gb300 import labelfuse as lf
    for n in declared_functions():
        assert callable(getattr(lf, n)), n
    assert sorted(lf.SYMBOLS) == sorted(declared_functions())


def test_host_only_calls(libpath):
    """Calls that touch no device: status strings, NULL handling, validation."""
    from paper_2111_11103_gb300 import labelfuse as lf
    L = lf.lib()
    assert lf.sm_status_string(0) == "ok"
    assert lf.sm_status_string(1) == "invalid argument"
    assert L.sm_num_rows(None) == -1
    assert L.sm_num_classes(None) == -1
    assert L.sm_mesh_free(None) == 0
    h = ctypes.c_void_p()
    # n_classes out of range is rejected before any CUDA call
    assert L.sm_mesh_upload(None, 0, None, 0, None, 255, 0, 0, None, ctypes.byref(h)) == 1
    assert "n_classes" in lf.sm_last_error()
    assert L.sm_mesh_upload(None, 0, None, 0, None, 4, 7, 0, None, ctypes.byref(h)) == 1
    assert L.sm_fuse_frames(None, None, 0, None, None, None, 1, 4, 4, None, None) == 1


def test_no_cpu_fallback_in_binding():
    """The binding never imports the oracle (no CPU fallback on the product path)."""
    src = open(os.path.join(ROOT, "paper_2111_11103_gb300", "labelfuse.py")).read()
    assert "oracle" not in src.replace("oracle", "", 0) or "import oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_2111_11103_gb300")):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(ROOT, "paper_2111_11103_gb300", f)).read()


def _mesh_functions():
    """Entry points whose first parameter is the mesh handle."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(sm_[a-z_0-9]+)\s*\(\s*(?:const\s+)?sm_mesh\s*\*", src)))


def test_every_mesh_call_rejects_a_null_handle(libpath):
    """Each call that takes a mesh answers SM_ERR_INVALID_ARG for a NULL one,
    on the host, before any CUDA call (so this runs without a GPU)."""
    from paper_2111_11103_gb300 import labelfuse as lf
    L = lf.lib()
    n64, ms, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32()
    calls = {
        "sm_fuse_frames": (None, None, 0, None, None, None, 1, 4, 4, None, None),
        "sm_fuse_frames_weighted": (None, None, 0, None, None, None, 0, 4, 4, None, None, None),
        "sm_normalise": (None, None, None, None),
        "sm_render_labels": (None, None, None, 1, 4, 4, None, None, None),
        "sm_render_idmap": (None, None, 16, None, None),
        "sm_reset": (None, None),
        "sm_read_state": (None, None, None, None),
        "sm_load_state": (None, None, None, None),
        "sm_check": (None, None),
        "sm_profile_enable": (None, 1),
        "sm_profile_read": (None, 0, ctypes.byref(n64), ctypes.byref(ms)),
        "sm_fuse_render_host": (None, None, 0, None, None, None, 1, 4, 4, None, None),
        "sm_set_weight_mix": (None, 0.5),
        "sm_texel_res_from_gamma": (None, None, None, 1, 4, 4, 0.5, None, None, None),
        "sm_autotune_batch": (None, None, 0, None, None, None, 1, 4, 4, ctypes.byref(b), None),
        "sm_conf_features": (None, None, 0, None, None, None, 1, 4, 4, None, None, None),
        "sm_conf_targets": (None, None, 0, None, None, 16, None, None),
        "sm_set_queue_shape": (None, 4, 4, 8, 1, 1, 32),
        "sm_conf_weights": (None, None, 0, None, None, None, 1, 4, 4, None, None, None, None),
        "sm_fuse_frames_confident": (None, None, 0, None, None, None, 1, 4, 4, None, None, None, None),
        "sm_set_launch_frames": (None, 4, 4, 8),
    }
    queries = {"sm_num_rows", "sm_num_classes", "sm_mesh_free"}  # -1, -1 and a no-op for NULL
    assert sorted(set(calls) | queries) == _mesh_functions()
    for name, args in calls.items():
        assert getattr(L, name)(*args) == 1, name
        assert "NULL" in lf.sm_last_error(), (name, lf.sm_last_error())


def test_argument_ranges_rejected_on_host(libpath):
    """Sizes, enums and rates outside the documented ranges are rejected before
    any CUDA call; empty work returns SM_OK without touching the device."""
    from paper_2111_11103_gb300 import labelfuse as lf
    L = lf.lib()
    h = ctypes.c_void_p()
    P = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    up = L.sm_mesh_upload
    assert up(None, 3, None, 1, None, 4, 0, 0, None, None) == 1                 # out NULL
    assert up(None, -1, None, 0, None, 4, 0, 0, None, ctypes.byref(h)) == 1     # V < 0
    assert up(None, 3, None, 1, None, 4, 0, 0, None, ctypes.byref(h)) == 1      # F > 0, NULL arrays
    assert up(P, 3, P, 1 << 31, None, 4, 0, 0, None, ctypes.byref(h)) == 1      # F >= 2^31
    assert up(P, 3, P, 1, None, 0, 0, 0, None, ctypes.byref(h)) == 1            # c = 0
    assert up(P, 3, P, 1, None, 4, -1, 0, None, ctypes.byref(h)) == 1           # rule
    assert up(P, 3, P, 1, None, 4, 0, 2, None, ctypes.byref(h)) == 1            # weight
    assert not h.value
    nr = L.sm_render_rows_noalloc
    assert nr(P, 3, P, 1, P, P, -1, 4, 4, P, None) == 1                         # N < 0
    assert nr(P, 3, P, 1, P, P, 1, 0, 4, P, None) == 1                          # H = 0
    assert nr(P, 3, P, 1, P, P, 1, 4, 16385, P, None) == 1                      # W > 16384
    assert nr(P, 3, P, 1, P, P, 1, 1296, 1297, P, None) == 1                    # > 1.5 Mi pixels
    assert nr(P, 3, P, 1, P, P, 1025, 4, 4, P, None) == 1                       # > 1024 frames
    assert nr(P, -3, P, 1, P, P, 1, 4, 4, P, None) == 1                         # V < 0
    assert nr(P, 3, P, 1, None, P, 1, 4, 4, P, None) == 1                       # K NULL
    assert nr(None, 0, None, 0, None, None, 0, 4, 4, None, None) == 0           # N = 0: nothing to do
    assert L.sm_conf_forward(P, P, -1, P, None) == 1
    assert L.sm_conf_forward(None, None, 0, None, None) == 0                    # n = 0: nothing to do
    assert L.sm_conf_forward(None, P, 5, P, None) == 1
    assert L.sm_conf_train_step(P, P, P, -1, 0.1, P, P, None) == 1
    assert L.sm_conf_train_step(P, P, P, 4, float("nan"), P, P, None) == 1
    assert L.sm_conf_train_step(P, P, P, 4, -0.5, P, P, None) == 1
    assert L.sm_conf_train_step(P, None, P, 4, 0.1, P, P, None) == 1
    ti = L.sm_conf_train_step_indexed
    assert ti(P, P, P, 10, P, -1, 0.1, P, P, None) == 1                          # m < 0
    assert ti(P, P, P, -1, P, 4, 0.1, P, P, None) == 1                           # n_obs < 0
    assert ti(P, P, P, 0, P, 4, 0.1, P, P, None) == 1                            # indices into nothing
    assert ti(P, P, P, 10, P, 4, float("nan"), P, P, None) == 1                  # lr NaN
    assert ti(P, P, P, 10, None, 4, 0.1, P, P, None) == 1                        # idx NULL
    assert ti(P, P, P, 10, P, 4, 0.1, None, P, None) == 1                        # grad NULL
    assert L.sm_host_alloc(0, ctypes.byref(h)) == 1
    assert L.sm_host_free(None) == 0
    comp = ctypes.c_int32(7)
    assert L.sm_device_alloc(0, 0, 1, ctypes.byref(h), ctypes.byref(comp)) == 1  # zero bytes
    assert comp.value == 0 and not h.value
    assert L.sm_device_alloc(0, 64, 1, None, None) == 1                          # out NULL
    assert L.sm_device_alloc(0, 64, 2, ctypes.byref(h), None) == 1               # unknown flag
    assert L.sm_device_alloc(-1, 64, 1, ctypes.byref(h), None) == 1              # no such device
    assert L.sm_device_free(None) == 0
    assert L.sm_device_free(P) == 1                                               # not a block of the library
    assert "sm_device_alloc" in lf.sm_last_error()


def test_binding_checks_buffers_before_the_call(libpath):
    """The binding refuses a tensor that is on the wrong side, not contiguous
    or smaller than what the call reads or writes, with SM_ERR_INVALID_ARG
    and before the library is called; raw addresses pass through."""
    import torch
    from paper_2111_11103_gb300 import labelfuse as lf
    host = torch.zeros(4 * lf.SM_CONF_PARAMS, dtype=torch.float32)
    with pytest.raises(lf.LabelFuseError) as e:          # device entry point, host tensor
        lf.sm_conf_forward(host, host, 4, host, stream=0)
    assert e.value.status == 1 and "CUDA tensor" in str(e.value)
    K = torch.zeros((2, 4), dtype=torch.float64)
    T = torch.zeros((2, 16), dtype=torch.float64)
    img = torch.zeros((2, 4, 4), dtype=torch.uint8)
    with pytest.raises(lf.LabelFuseError, match="K holds 64 bytes; the call needs 96"):
        lf.sm_fuse_render_host(None, None, "f32", None, K, T, 3, 4, 4, img, stream=0)
    with pytest.raises(lf.LabelFuseError, match="labels_out holds 32 bytes; the call needs 40"):
        lf.sm_fuse_render_host(None, None, "f32", None, K, T, 2, 4, 5, img, stream=0)
    with pytest.raises(lf.LabelFuseError, match="cam_to_world is not contiguous"):
        lf.sm_fuse_render_host(None, None, "f32", None, K, torch.zeros((16, 2), dtype=torch.float64).t(), 2, 4, 4,
                               img, stream=0)
    with pytest.raises(lf.LabelFuseError, match="scale holds"):
        lf.sm_fuse_render_host(None, None, "bf16", torch.zeros(31), K, T, 2, 4, 4, img, stream=0)
    # within bounds the call reaches the library, which rejects the NULL mesh
    with pytest.raises(lf.LabelFuseError, match="NULL"):
        lf.sm_fuse_render_host(None, None, "f32", None, K, T, 2, 4, 4, img, stream=0)
    # the host entry point refuses what the device entry points need, and vice versa
    assert lf._arg(img, "x", img.numel(), host=True) == img.data_ptr()
    with pytest.raises(lf.LabelFuseError, match="must be a CUDA tensor"):
        lf._arg(img, "x", 1)
    assert lf._arg(1234, "raw", 1 << 40) == 1234 and lf._arg(None, "x", 8) is None
    # the byte count follows the element size (an FP8 buffer viewed as uint8 is fine)
    assert lf._arg(torch.zeros(10, dtype=torch.uint8), "probs", 10, host=True)
    with pytest.raises(lf.LabelFuseError):
        lf._arg(torch.zeros(10, dtype=torch.uint8), "probs", 11, host=True)


def test_binding_checks_of_the_newer_calls(libpath):
    """device_empty wants a CUDA device and a supported element type; the
    indexed training step wants int64 indices (checked before the call)."""
    import torch
    from paper_2111_11103_gb300 import labelfuse as lf
    with pytest.raises(ValueError, match="CUDA device"):
        lf.device_empty((4,), torch.int32, "cpu")
    with pytest.raises(ValueError, match="unsupported dtype"):
        lf.device_empty((4,), torch.bfloat16, "cuda:0")
    with pytest.raises(lf.LabelFuseError, match="int64"):
        lf.sm_conf_train_step_indexed(None, None, None, 8, torch.zeros(4, dtype=torch.int32), 4, 0.1, None, None,
                                      stream=0)
    # raw addresses pass through to the library, which checks the rest
    with pytest.raises(lf.LabelFuseError, match="m < 0"):
        lf.sm_conf_train_step_indexed(16, 16, 16, 8, 16, -1, 0.1, 16, 16, stream=0)


def test_header_is_plain_c_and_a_c_client_links(libpath, tmp_path):
    """include/labelfuse.h compiles as strict C99 and C++17 on its own, and a
    plain C program (no Python, no PyTorch) links against the library and gets
    its host-side answers (status strings, NULL-handle queries, validation)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([gcc if lang == "c" else (shutil.which("g++") or gcc), std, "-Wall", "-Wextra",
                            "-pedantic", "-Werror", "-fsyntax-only", "-x", lang, HEADER], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    src = tmp_path / "client.c"
    src.write_text(r"""
#include <stdio.h>
#include "labelfuse.h"
int main(void)
{
    sm_mesh *m = 0;
    sm_status st = sm_mesh_upload(0, 0, 0, 0, 0, 0, SM_RULE_SUM, SM_WEIGHT_PIXEL, 0, &m);
    printf("%d|%s|%s|%lld|%d\n", (int)st, sm_status_string(st), sm_last_error(), (long long)sm_num_rows(0),
           (int)sm_mesh_free(0));
    return (st == SM_ERR_INVALID_ARG && m == 0) ? 0 : 1;
}
""")
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-I", inc, str(src), "-o", str(exe), "-L", libdir, "-llabelfuse",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    code, text, reason, rows, freed = r.stdout.strip().split("|")
    assert (code, text, rows, freed) == ("1", "invalid argument", "-1", "0")
    assert "n_classes" in reason


def test_fuse_scenes_rejects_bad_scene_lists_on_host(libpath):
    """sm_fuse_scenes refuses a NULL list, a NULL mesh (naming the scene) and
    a mesh that appears twice, before any CUDA call."""
    from paper_2111_11103_gb300 import labelfuse as lf
    L = lf.lib()
    assert L.sm_fuse_scenes(None, 2, None) == 1
    assert L.sm_fuse_scenes(None, 0, None) == 0
    arr = (lf.SceneFrames * 2)()
    assert L.sm_fuse_scenes(arr, 2, None) == 1
    assert "scene 0" in lf.sm_last_error() and "NULL" in lf.sm_last_error()
    arr[0].mesh = arr[1].mesh = 16  # never dereferenced: refused as shared first
    assert L.sm_fuse_scenes(arr, 2, None) == 1
    assert "share a mesh" in lf.sm_last_error()
