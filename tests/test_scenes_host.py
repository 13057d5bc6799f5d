"""Host-side checks of the side-by-side scene runner (no GPU needed: both
cases return before any stream or library call)."""
import pytest
import torch

from paper_2111_11103_gb300 import scenes


def _job(mesh):
    z = torch.zeros(1)
    return scenes.SceneJob(mesh=mesh, probs=z, K=z, cam_to_world=z, H=1, W=1)


def test_a_mesh_may_appear_in_one_job_only():
    with pytest.raises(ValueError, match="one job only"):
        scenes.fuse_scenes([_job(1), _job(2), _job(1)])


def test_no_jobs_is_a_no_op():
    assert scenes.fuse_scenes([]) is None
