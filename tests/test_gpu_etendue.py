"""Etendue comparison (Fig. 7 of the paper) through the lens-train printer: runs end to end
on the GPU and returns valid voxel error rates."""
import pytest

pytestmark = pytest.mark.gpu


def test_etendue_experiment_runs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import etendue as E
    r = E.etendue_experiment(16.0, iters=5)
    assert 0 < r["rays_in_resin_13"] <= r["rays_total_13"]
    for k in ("chief_ray_model", "thirteen_ray_model"):
        assert 0.0 <= r[k]["ver_in_13_ray_printer"] <= 1.0
