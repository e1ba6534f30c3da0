"""Learned warm start: trained on pairs the plain optimiser itself produces, the network's
projections start the projection-space iteration closer to the optimum than the same
iteration started from the method's own first projections max(0, A^T f).

Workload: the 128^3 warm-start optics (pupil 100 mm, f/4, 4 rays/pixel, vial 6/1 mm,
mu 0.05) on a 64x64x32 grid with 128x32 pixels and 64 angles, seeded CSG targets.
"""
import numpy as np
import pytest
import torch

from paper_2211_03516_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

SMALL = I.WORKLOADS["warmstart_128cube_180ang_4rays"].scaled(
    nx=64, ny=64, nz=32, voxel_mm=0.2, nu=128, nv=32, pixel_u_mm=0.1, pixel_v_mm=0.2, n_angles=64)


@pytest.fixture(scope="module")
def trained():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import unet as U
    from paper_2211_03516_gb300 import vamrt as V
    from paper_2211_03516_gb300 import warmstart as WS
    P = V.Projector.from_workload(SMALL, I.workload_pupil(SMALL))
    pairs = WS.make_pairs(P, SMALL, range(32), osmo_iters=15)
    net = U.UNet3D(DEV, seed=0)
    losses = WS.train(net, pairs, epochs=10, lr=1e-3)
    return P, net, WS, losses


def test_training_lowers_the_loss(trained):
    _, _, _, losses = trained
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0]


def test_warm_start_beats_the_method_without_it(trained):
    P, net, WS, _ = trained
    rows = WS.compare(P, net, SMALL, range(10000, 10004), plain_iters=15, cont_iters=6, step=0.5)
    assert len(rows) == 4
    warm_first = np.mean([r["warm_ver"][0] for r in rows])
    cold_first = np.mean([r["cold_ver"][0] for r in rows])
    warm_best = np.mean([min(r["warm_ver"]) for r in rows])
    cold_best = np.mean([min(r["cold_ver"]) for r in rows])
    plain_at6 = np.mean([r["plain_ver"][5] for r in rows])
    # the network's projections print better than A^T f, and after the same number of
    # iterations the warm-started run is ahead of both the cold start and the plain loop
    assert warm_first < 0.9 * cold_first
    assert warm_best < cold_best
    assert warm_best < plain_at6
    # the adjoint-driven continuation (thresholded-loss Adam steps, BF16 storage) from the
    # network's projections stays ahead of the same continuation from A^T f
    warm_loss = np.mean([min(r["warm_loss_ver"]) for r in rows])
    cold_loss = np.mean([min(r["cold_loss_ver"]) for r in rows])
    assert warm_loss < cold_loss
