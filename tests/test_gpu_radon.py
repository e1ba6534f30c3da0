"""Radon-method baseline (Sec. 2.3): the CUDA Ram-Lak filter and the Radon projections
against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import radon as RD
from oracle import vam_oracle as O
from paper_2211_03516_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import vamrt
    return vamrt


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("rows,nu", [(37, 256), (5, 1), (3, 17), (2, 4096), (90, 64)])
def test_ramlak_filter_matches_oracle(V, rows, nu):
    rng = np.random.default_rng(rows * 7 + nu)
    p = rng.random((rows, nu)).astype(np.float32)
    tau = 0.1
    ref = RD.ramlak_filter(p, tau)
    x = torch.from_numpy(p).to(DEV)
    q = V.ramlak_filter(x, tau)
    qc = V.ramlak_filter(x, tau, clamp=True)
    torch.cuda.synchronize()
    assert rel_l2(q.cpu().numpy(), ref) <= FP32_TOL
    assert rel_l2(qc.cpu().numpy(), np.maximum(ref, 0.0)) <= FP32_TOL
    assert float(qc.min()) >= 0.0
    V.ramlak_filter(x, tau, clamp=True, out=x)            # in place
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), qc.cpu().numpy())


def test_ramlak_filter_bad_arguments(V):
    x = torch.zeros((2, 5000), device=DEV)
    with pytest.raises(V.VamrtError):
        V.ramlak_filter(x, 0.1)                                 # nu beyond 4096
    with pytest.raises(V.VamrtError):
        V.ramlak_filter(torch.zeros((2, 8), device=DEV), 0.0)    # pitch
    e = torch.zeros((0, 8), device=DEV)
    assert V.ramlak_filter(e, 0.1).shape == (0, 8)              # no rows: nothing to do


def test_radon_projections_match_oracle(V):
    """R f on the Radon geometry (parallel chief rays, no refraction or attenuation),
    filtered and clipped, against the oracle's projection on the same geometry and its
    filter."""
    from paper_2211_03516_gb300 import radon as R
    w = I.TINY
    wr = I.radon_workload(w)
    pupil = I.workload_pupil(wr)
    f = I.make_target(w)
    P = V.Projector.from_workload(wr, pupil)
    g = R.radon_projections(P, torch.from_numpy(f).to(DEV), w.pixel_u_mm)
    torch.cuda.synchronize()
    ref = RD.ramlak_filter(O.adjoint(wr, f, pupil), w.pixel_u_mm, clamp=True)
    assert rel_l2(g.cpu().numpy(), ref) <= FP32_TOL
    P.close()


def test_radon_baseline_voxel_error_rates(V):
    """On its own (ideal) printer the Radon method reconstructs the target (filtered
    backprojection); in the refracting ray-traced printer its dose is worse."""
    from paper_2211_03516_gb300 import radon as R
    w = I.TINY
    P = V.Projector.from_workload(w, I.workload_pupil(w))
    f = torch.from_numpy(I.make_target(w)).to(DEV)
    r = R.radon_baseline(P, w, f)
    assert 0.0 <= r["ver_ideal_radon_printer"] < 0.05
    assert r["ver_ideal_radon_printer"] < r["ver_ray_traced_printer"] <= 1.0
    P.close()
