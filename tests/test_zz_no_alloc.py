"""vamrt_forward_dose_static: the dose operator for callers that cannot allocate.

The entry point runs the dose kernels with a statically allocated 16 MiB accumulator
instead of the projector's scratch volume, so a caller whose device memory is owned by
another allocator (or who must not allocate where it calls) can still compute doses.
It is called here through the C ABI and checked against vamrt_forward_dose on the same
input, on two calls in a row (the shared array keeps the previous call's sums, so the
second call shows that each call clears it).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2211_03516_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5          # the tolerance the operator parity tests use
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def V():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_03516_gb300 import vamrt
    L = vamrt.lib()
    L.vamrt_forward_dose_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p]
    L.vamrt_forward_dose_static.restype = ctypes.c_int
    return vamrt


def rel_l2(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def static_dose(V, P, proj, dose, accumulate=False):
    dt = {torch.float32: V.VAMRT_F32, torch.bfloat16: V.VAMRT_BF16}
    st = V.lib().vamrt_forward_dose_static(P.handle, proj.data_ptr(), dt[proj.dtype], dose.data_ptr(),
                                           dt[dose.dtype], V.VAMRT_ACCUMULATE if accumulate else 0,
                                           torch.cuda.current_stream().cuda_stream)
    return st


WORKLOADS = {
    "tiny": I.TINY,
    "refracting_ragged": I.TINY.scaled(nx=33, ny=34, nz=23, voxel_mm=0.4, nu=37, nv=23, pixel_u_mm=0.38,
                                       pixel_v_mm=0.41, n_angles=10, f_number=3.5, pupil_pattern="sunflower",
                                       rays_per_pixel=4, pupil_mm=60.0),
    "warm_start_128": I.WORKLOADS["warmstart_128cube_180ang_4rays"].scaled(n_angles=30),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_static_dose_matches_forward_dose_twice(V, name):
    w = WORKLOADS[name]
    P = V.Projector.from_workload(w, I.workload_pupil(w))
    for seed in (5, 6):      # two calls in a row, different inputs
        g = torch.from_numpy(I.random_projections(w, seed=seed)).to(DEV)
        ref = P.forward_dose(g)
        out = torch.full(w.vol_shape, float("nan"), device=DEV)
        assert static_dose(V, P, g, out) == V.VAMRT_OK, V.lib().vamrt_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel_l2(out, ref) <= FP32_TOL


def test_static_dose_leaves_device_memory_unchanged(V):
    """The entry point's reason to exist: two calls in a row change neither the device's
    free memory (cudaMemGetInfo) nor what torch's allocator holds."""
    w = WORKLOADS["refracting_ragged"]
    P = V.Projector.from_workload(w, I.workload_pupil(w))
    g = torch.from_numpy(I.random_projections(w, seed=13)).to(DEV)
    ref = P.forward_dose(g)
    out = torch.empty(w.vol_shape, device=DEV)
    torch.cuda.synchronize()
    free0, held0 = torch.cuda.mem_get_info(DEV)[0], torch.cuda.memory_allocated(DEV)
    for _ in range(2):
        assert static_dose(V, P, g, out) == V.VAMRT_OK, V.lib().vamrt_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(DEV)[0] == free0
    assert torch.cuda.memory_allocated(DEV) == held0
    assert rel_l2(out, ref) <= FP32_TOL


def test_static_dose_accumulate_and_bf16(V):
    w = WORKLOADS["refracting_ragged"]
    P = V.Projector.from_workload(w, I.workload_pupil(w))
    g = torch.from_numpy(I.random_projections(w, seed=9)).to(DEV)
    ref = P.forward_dose(g)
    out = ref.clone()
    assert static_dose(V, P, g, out, accumulate=True) == V.VAMRT_OK
    assert rel_l2(out, 2 * ref) <= FP32_TOL
    g16 = g.to(torch.bfloat16)
    ref16 = P.forward_dose(g16, dose_dtype=torch.bfloat16)
    out16 = torch.empty(w.vol_shape, device=DEV, dtype=torch.bfloat16)
    assert static_dose(V, P, g16, out16) == V.VAMRT_OK
    assert rel_l2(out16, ref16) <= 2e-3


def test_static_dose_rejects_grids_beyond_the_array(V):
    w = I.MID.scaled(n_angles=2, nu=32, nv=32, rays_per_pixel=1, pupil_pattern="chief", f_number=float("inf"))
    P = V.Projector.from_workload(w, I.workload_pupil(w))
    g = torch.ones(w.proj_shape, device=DEV)
    out = torch.zeros(w.vol_shape, device=DEV)
    assert static_dose(V, P, g, out) == V.VAMRT_EINVAL
    assert b"too large for the static accumulator" in V.lib().vamrt_last_error()
    assert V.lib().vamrt_forward_dose_static(None, None, 0, None, 0, 0, None) == V.VAMRT_EINVAL
