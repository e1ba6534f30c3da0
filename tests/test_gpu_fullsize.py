"""Parity at the full sizes of the large workloads, in the launch configuration the
benchmark times, against the FP64 oracle on outputs it can compute one by one.

  large print   768 x 768 x 1024 voxels (0.05 mm), 1000 angles, 1024^2 pixels, f/2.8, 4 rays
  tall build    384 x 384 x 512 voxels (0.08 mm), 720 angles, 384 x 512 pixels, 8 rays,
                projections and dose stored in BF16 (FP32 sums)
  mid           256^3 voxels, 360 angles, 256^2 pixels, 16 stratified rays (dense dose)

Checks: sampled projection pixels (the oracle traces those pixels' rays only); the dose
of sparse projections (the oracle lists each pixel's contributions); the dose of a dense
band of one angle (a one-angle projector: the same ray table, one rotation); the adjoint
identity over whole random volumes.  Tolerances: 1e-5 relative L2 (FP32), 2e-3 for
BF16-stored outputs, 1e-3 for FP32 results of BF16-stored inputs.
"""
import numpy as np
import pytest
import torch

from oracle import vam_oracle as O
from paper_2211_03516_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_OUT_TOL = 2e-3
BF16_IN_TOL = 1e-3
DEV = torch.device("cuda:0")
LARGE = I.WORKLOADS["large_768x768x1024_1000ang_4rays"]
TALL = I.WORKLOADS["tall_384x384x512_720ang_8rays"]


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import vamrt
    return vamrt


def sampled_pixels(y, w, rng, n_hit=40, n_any=8):
    """Pixels whose rays cross the part, plus a few arbitrary ones."""
    hit = torch.nonzero(y > 0.05 * y.max()).cpu().numpy()
    pick = hit[rng.choice(len(hit), n_hit, replace=False)]
    return np.concatenate([pick, np.stack([rng.integers(0, s, n_any) for s in w.proj_shape], 1)])


def check_sparse_dose(V, P, w, pupil, dose_dtype, tol, seed):
    """Dose of projections nonzero at 48 seeded pixels: at the voxels the oracle's rays
    reach, against its FP64 sums; zero elsewhere."""
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, s, 48) for s in w.proj_shape], 1)
    vals = (0.5 + rng.integers(0, 128, 48) / 128.0).astype(np.float32)     # exact in BF16 too
    g = torch.zeros(w.proj_shape, device=DEV)
    g[tuple(torch.from_numpy(pix.T).to(DEV))] = torch.from_numpy(vals).to(DEV)
    d = P.forward_dose(g, dose_dtype=dose_dtype).float().view(-1)
    idx, ref = O.forward_pixels(w, pupil, [tuple(p) for p in pix], vals.astype(np.float64))
    got = d[torch.from_numpy(idx).to(DEV)].cpu().numpy()
    assert rel_l2(got, ref) <= tol
    outside = d.clone()
    outside[torch.from_numpy(idx).to(DEV)] = 0
    assert float(outside.abs().max()) == 0.0


def check_dense_band(V, w, pupil, k, rows, seed, tol=FP32_TOL, dose_dtype=torch.float32):
    """Dense dose of one angle's band of pixel rows, through a one-angle projector (the same
    ray table; only the rotation differs), against the oracle's dense FP64 dose."""
    ang = I.default_angles(w.n_angles)[k:k + 1]
    w1 = w.scaled(n_angles=1)
    P1 = V.Projector.from_workload(w1, pupil, angles_rad=ang)
    g = np.zeros(w1.proj_shape, np.float32)
    g[0, rows[0]:rows[1], :] = np.random.default_rng(seed).random((rows[1] - rows[0], w.nu), dtype=np.float32)
    d = P1.forward_dose(torch.from_numpy(g).to(DEV), dose_dtype=dose_dtype).float().cpu().numpy()
    ref = O.forward(w1, g, pupil, angles=ang)
    assert rel_l2(d, ref) <= tol


# ---- large print: 768 x 768 x 1024, 1000 angles, 1024^2 pixels, 4 rays ------------------
@pytest.fixture(scope="module")
def large(V):
    w = LARGE
    pupil = I.workload_pupil(w)
    P = V.Projector.from_workload(w, pupil)
    f = I.make_target(w)
    return w, pupil, P, f


def test_large_sample_count_and_adjoint_identity(V, large):
    w, pupil, P, _ = large
    n = P.sample_count()
    assert 3.0e12 < n < 6.0e12
    Vr = torch.from_numpy(I.random_volume(w, seed=21)).to(DEV)
    g = torch.from_numpy(I.random_projections(w, seed=22)).to(DEV)
    lhs = torch.sum(P.forward_dose(g).double() * Vr.double()).item()
    rhs = torch.sum(g.double() * P.adjoint(Vr).double()).item()
    assert abs(lhs - rhs) <= FP32_TOL * abs(rhs)


def test_large_sampled_pixels_match_oracle(V, large):
    w, pupil, P, f = large
    y = P.adjoint(torch.from_numpy(f).to(DEV))
    pick = sampled_pixels(y, w, np.random.default_rng(7))
    got = y[tuple(torch.from_numpy(pick.T).to(DEV))].cpu().numpy()
    ref = O.adjoint_pixels(w, f, pupil, [tuple(p) for p in pick])
    assert rel_l2(got, ref) <= FP32_TOL
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    assert np.all(np.abs(got[big] - ref[big]) <= 1e-4 * np.abs(ref[big]))


def test_large_sparse_dose_matches_oracle(V, large):
    w, pupil, P, _ = large
    check_sparse_dose(V, P, w, pupil, torch.float32, FP32_TOL, seed=5)


def test_large_dense_band_dose_matches_oracle(V, large):
    w, pupil, _, _ = large
    check_dense_band(V, w, pupil, k=137, rows=(480, 544), seed=6)


# ---- tall build: 384 x 384 x 512, 720 angles, 8 rays, BF16 storage ----------------------
@pytest.fixture(scope="module")
def tall(V):
    w = TALL
    pupil = I.workload_pupil(w)
    P = V.Projector.from_workload(w, pupil)
    f = I.make_target(w)
    return w, pupil, P, f


def test_tall_bf16_projection_sampled_pixels(V, tall):
    """BF16-stored projections of the (exactly representable) binary target, on 2000
    sampled pixels: within 2e-3 relative L2 of the FP64 oracle (BF16 rounding alone is
    ~1.1e-3 RMS; a few dozen samples near a power of two can exceed 2e-3 by themselves), and
    every value within one BF16 step of the oracle's (the FP32 sum rounds to a neighbour)."""
    w, pupil, P, f = tall
    y = P.adjoint(torch.from_numpy(f).to(DEV, torch.bfloat16), proj_dtype=torch.bfloat16)
    pick = sampled_pixels(y.float(), w, np.random.default_rng(8), n_hit=1800, n_any=200)
    got = y[tuple(torch.from_numpy(pick.T).to(DEV))].float().cpu().numpy()
    ref = O.adjoint_pixels(w, f, pupil, [tuple(p) for p in pick])
    assert rel_l2(got, ref) <= BF16_OUT_TOL
    ulp = np.exp2(np.floor(np.log2(np.maximum(np.abs(ref), 1e-30))) - 7)
    assert np.all(np.abs(got - ref) <= ulp * (1 + 1e-3) + 1e-30)


def test_tall_gradient_from_bf16_volume_sampled_pixels(V, tall):
    """A^T of a BF16-stored volume (the backward of the dose operator on a BF16 dL/dD), kept
    in FP32: the oracle sees the same BF16-rounded values."""
    w, pupil, P, _ = tall
    v16 = torch.from_numpy(I.random_volume(w, seed=31)).to(DEV, torch.bfloat16)
    y = P.adjoint(v16, proj_dtype=torch.float32)
    pick = np.stack([np.random.default_rng(9).integers(0, s, 48) for s in w.proj_shape], 1)
    got = y[tuple(torch.from_numpy(pick.T).to(DEV))].cpu().numpy()
    ref = O.adjoint_pixels(w, v16.float().cpu().numpy(), pupil, [tuple(p) for p in pick])
    assert rel_l2(got, ref) <= BF16_IN_TOL


def test_tall_bf16_sparse_dose(V, tall):
    w, pupil, P, _ = tall
    check_sparse_dose(V, P, w, pupil, torch.bfloat16, BF16_OUT_TOL, seed=10)


def test_tall_dense_band_dose_fp32_and_bf16(V, tall):
    w, pupil, _, _ = tall
    check_dense_band(V, w, pupil, k=301, rows=(200, 264), seed=11)
    check_dense_band(V, w, pupil, k=301, rows=(200, 264), seed=11, tol=BF16_OUT_TOL, dose_dtype=torch.bfloat16)


# ---- mid: a dense dose of whole angles ----------------------------------------------------
def test_mid_dense_dose_of_two_angles(V):
    """Every pixel of two angles of the 256^3 workload (one-angle projectors)."""
    w = I.MID
    pupil = I.workload_pupil(w)
    for k in (0, 97):
        check_dense_band(V, w, pupil, k=k, rows=(0, w.nv), seed=12 + k)
