"""vamrt_optimize in VAMRT_OPT_GRADIENT mode (the differentiable path driven through the C
ABI: projected Adam steps on the thresholded dose loss from caller-supplied starting
projections) against the FP64 oracle's reading of the same continuation
(oracle/osmo.py: threshold_adam).

Adam scales each pixel's step by its own gradient's magnitude: the first step is
lr * sign(gradient).  A pixel whose gradient is zero or within rounding of zero (a ray
that grazes the footprint of a voxel with a nonzero loss gradient at a trilinear weight
of ~1e-8) may step by lr in one precision and not at all in the other, so after a step
the projections are compared exactly where the oracle's gradient is well above rounding
and elsewhere checked to have moved by at most lr (the first Adam step's magnitude is
lr |m^| / sqrt(v^) <= lr) and to stay non-negative.  Zeroing every gradient below 1e-6 of
the largest in the oracle's own run moves its five-iteration losses by 0.4 % and its
projections by 0.07 %, so the trajectories are held to 2e-2.
"""
import numpy as np
import pytest
import torch

from oracle import osmo as OS
from oracle import vam_oracle as O
from paper_2211_03516_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
FP32_TOL = 1e-5
D_L, D_H, STEP = 0.8, 1.0, 0.8


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import vamrt
    w = I.TINY
    pupil = I.workload_pupil(w)
    P = vamrt.Projector.from_workload(w, pupil)
    f = I.make_target(w)
    g0 = np.maximum(0.0, O.adjoint(w, f, pupil))
    return dict(w=w, pupil=pupil, P=P, f=f, g0=g0, vamrt=vamrt)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def oracle_run(s, n_iter):
    w, pupil = s["w"], s["pupil"]
    return OS.threshold_adam(s["f"], s["g0"], lambda x: O.adjoint(w, x, pupil), lambda y: O.forward(w, y, pupil),
                             n_iter=n_iter, step=STEP, d_l=D_L, d_h=D_H)


def test_gradient_mode_first_step_matches_oracle(setup):
    s = setup
    w, pupil, f = s["w"], s["pupil"], s["f"]
    res = s["P"].optimize(gpu(f), proj=gpu(s["g0"]), mode="gradient", max_iter=1, tol=0.0, step=STEP,
                          d_l=D_L, d_h=D_H)
    g_ref, D_ref, L_ref = oracle_run(s, 1)
    # the scaled start, its dose and loss: the FP32 path's parity
    np.testing.assert_allclose(res["errors"], L_ref, rtol=FP32_TOL)
    assert rel_l2(res["dose"].cpu().numpy(), D_ref) <= FP32_TOL
    # the first step: g1 = max(0, g - lr sign(grad)) with g = g0 / mean_P(A g0)
    Ds = O.forward(w, s["g0"], pupil)
    gs = s["g0"] / Ds[f > 0.5].mean()
    lr = STEP * gs[gs > 0].mean()
    _, G = OS.threshold_loss(D_ref, f, D_L, D_H)
    grad = O.adjoint(w, G, pupil)
    g1 = res["proj"].cpu().numpy().astype(np.float64)
    clear = np.abs(grad) > 1e-3 * np.abs(grad).max()
    assert clear.sum() > 0.5 * (grad != 0).sum()
    assert rel_l2(g1[clear], g_ref[clear]) <= FP32_TOL
    # elsewhere: a step of at most lr, never below zero
    rest = ~clear
    assert (np.abs(g1[rest] - gs[rest]) <= lr * (1 + 1e-5) + 1e-6 * gs.max()).all()
    assert (g1 >= 0).all()


def test_gradient_mode_follows_oracle_over_iterations(setup):
    """Five iterations: the loss and voxel-error-rate trajectories follow the oracle's
    (aggregates over the whole volume, so the few pixels whose step differs leave them
    within 2e-2), and the loss falls."""
    s = setup
    f = s["f"]
    n = 5
    res = s["P"].optimize(gpu(f), proj=gpu(s["g0"]), mode="gradient", max_iter=n, tol=0.0, step=STEP,
                          d_l=D_L, d_h=D_H)
    g_ref, D_ref, L_ref = oracle_run(s, n)
    assert res["iterations"] == n
    np.testing.assert_allclose(res["errors"], L_ref, rtol=2e-2)
    assert res["errors"][-1] < 0.5 * res["errors"][0]
    Z, Y, X = I.voxel_centres(s["w"])
    v_ref, _ = OS.voxel_error_rate(D_ref, f, X ** 2 + Y ** 2 <= s["w"].r_inner_mm ** 2)
    assert abs(res["vers"][-1] - v_ref) <= 2e-2 * max(v_ref, 1e-3)
    assert rel_l2(res["proj"].cpu().numpy(), g_ref) <= 2e-2


def test_gradient_mode_bf16_storage_and_stop(setup):
    """BF16-stored projections and dose: the loss still falls, the projections stay BF16 and
    non-negative; a voxel-error-rate tolerance stops the run early."""
    s = setup
    f = s["f"]
    res = s["P"].optimize(gpu(f), proj=gpu(s["g0"], torch.bfloat16), dose_dtype=torch.bfloat16, mode="gradient",
                          max_iter=6, tol=0.0, step=STEP, d_l=D_L, d_h=D_H)
    assert res["proj"].dtype == torch.bfloat16 and res["dose"].dtype == torch.bfloat16
    assert (res["proj"].float() >= 0).all()
    assert np.isfinite(res["errors"]).all() and res["errors"][-1] < res["errors"][0]
    goal = float(res["vers"][2]) + 1e-3      # ~180 resin voxels: the scatter's summation order may move a few
    res2 = s["P"].optimize(gpu(f), proj=gpu(s["g0"], torch.bfloat16), dose_dtype=torch.bfloat16, mode="gradient",
                           max_iter=6, tol=goal, step=STEP, d_l=D_L, d_h=D_H)
    assert res2["converged"] and res2["iterations"] <= 3


def test_gradient_mode_rejects_bad_arguments(setup):
    s = setup
    V, P, f = s["vamrt"], s["P"], s["f"]
    with pytest.raises(V.VamrtError):
        P.optimize(gpu(f), proj=gpu(s["g0"], torch.float16), mode="gradient", max_iter=1)
    with pytest.raises(V.VamrtError):
        P.optimize(gpu(f), proj=gpu(s["g0"]), mode="gradient", max_iter=1, d_l=1.0, d_h=0.5)
    with pytest.raises(V.VamrtError):
        P.optimize(gpu(f), proj=torch.zeros(s["w"].proj_shape, device=DEV), mode="gradient", max_iter=1)
