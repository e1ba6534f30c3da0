"""Radon-method baseline (Sec. 2.3) on the GPU: the projections a Radon-based printer
computes -- parallel-beam Radon transform of each z-slice, Ram-Lak filter, negatives
clipped -- and the dose they deliver in the ray-traced printer, for comparison with the
3D-ray-traced optimiser (the paper's central comparison).  Every step runs in the CUDA
library: the Radon transform is the projection kernel on the Radon geometry
(`inputs.radon_workload`), the filter `vamrt_ramlak_filter`, the dose the dose kernel."""
from __future__ import annotations

import torch

from . import inputs as I
from . import vamrt as V


def radon_projections(P_radon: V.Projector, target: torch.Tensor, pixel_mm: float) -> torch.Tensor:
    """max(0, RamLak(R f)): R = the projection on the Radon geometry (parallel chief rays,
    no refraction or attenuation), filtered along u with detector pitch pixel_mm."""
    y = P_radon.adjoint(target)
    return V.ramlak_filter(y, pixel_mm, clamp=True, out=y)


def radon_baseline(P: V.Projector, w, target: torch.Tensor) -> dict:
    """Voxel error rate of the Radon-method projections dosed by the ideal Radon printer
    (the geometry they assume) and by the ray-traced printer P (refraction at the vial,
    the pupil's non-telecentricity and etendue, attenuation)."""
    wr = I.radon_workload(w)
    P_radon = V.Projector.from_workload(wr, I.workload_pupil(wr))
    try:
        g = radon_projections(P_radon, target, w.pixel_u_mm)
        d_ideal = P_radon.forward_dose(g)
        d_real = P.forward_dose(g)
        return {"ver_ideal_radon_printer": P_radon.voxel_error_rate(d_ideal, target)[0],
                "ver_ray_traced_printer": P.voxel_error_rate(d_real, target)[0],
                "projections": g}
    finally:
        P_radon.close()
