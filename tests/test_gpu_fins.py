"""Fin-part comparison (Radon method vs ray-traced optimiser in the non-telecentric
printer) on a 3-fin part: it runs end to end on the GPU and returns valid counts."""
import pytest

pytestmark = pytest.mark.gpu


def test_fins_experiment_three_fins():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import fins as F
    r = F.fins_experiment(3, iters=10)
    for k in ("ray_traced", "radon"):
        assert 0.0 <= r[k]["ver"] <= 1.0
        assert 0 <= r[k]["fins_formed"] <= 3 and len(r[k]["per_fin"]) == 3
    assert r["ray_traced"]["ver"] < r["radon"]["ver"]


@pytest.mark.parametrize("n_fins,n_angles", [(9, 12), (18, 6)])
def test_fins_geometry_operators_match_oracle(n_fins, n_angles):
    """The fin printer of Sec. 2.6.1 at its full height (216 planes for 9 fins, 404 for 18:
    chief rays up to 12 and 23 degrees off the optical axis in air), on fewer angles: the
    projection of the fin part and the dose of random projections match the FP64 oracle
    (1e-5 relative L2), and the ray table's sample count matches exactly."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from oracle import vam_oracle as O
    from paper_2211_03516_gb300 import inputs as I
    from paper_2211_03516_gb300 import vamrt as V

    w = I.fins_workload(n_fins).scaled(n_angles=n_angles)
    pupil = I.workload_pupil(w)
    P = V.Projector.from_workload(w, pupil)
    assert P.sample_count() == O.sample_count(w, pupil)
    f = I.make_target(w)
    y = P.adjoint(torch.from_numpy(f).to("cuda")).cpu().numpy()
    g = I.random_projections(w, seed=4)
    d = P.forward_dose(torch.from_numpy(g).to("cuda")).cpu().numpy()
    y_ref = O.adjoint(w, f, pupil)
    d_ref = O.forward(w, g, pupil)

    def rel(a, b):
        return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))

    assert rel(y, y_ref) <= 1e-5
    assert rel(d, d_ref) <= 1e-5
    # the steepest chief ray in air: atan(half the image height / pupil distance)
    assert np.degrees(np.arctan(0.5 * w.nv * w.pixel_v_mm / w.pupil_mm)) > (11.0 if n_fins == 9 else 22.0)
