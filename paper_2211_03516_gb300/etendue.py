"""Etendue comparison of Sec. 3 (Fig. 7): in the telecentric printer of Sec. 2.6.2 (a 4f
lens relay with a 2.5 mm or 16 mm iris), projections optimised with a chief-ray-only model
of the printer (the zero-etendue assumption of Radon-based methods) against projections
optimised with 13 rays per pixel traced through the lenses, both dosed by the 13-ray
printer.  Every projection and dose comes from the CUDA library."""
from __future__ import annotations

import torch

from . import inputs as I
from . import vamrt as V


def _optimise(P, f, iters, beta, mu):
    model, prev = f.clone(), f.clone()
    for _ in range(iters):
        res = P.optimize(f, model=model, prev_model=prev, max_iter=1, tol=0.0, step=beta, momentum=mu)
    return res["proj"]


def etendue_experiment(iris_diameter_mm: float, seed: int = 0, iters: int = 20, beta: float = 4.0,
                       mu: float = 0.5, kind: str = "csg") -> dict:
    w13 = I.etendue_workload(iris_diameter_mm, "hex13")
    w1 = I.etendue_workload(iris_diameter_mm, "chief")
    P13 = V.Projector.from_workload(w13, I.workload_pupil(w13))
    P1 = V.Projector.from_workload(w1, I.workload_pupil(w1))
    try:
        f = torch.from_numpy(I.make_target(w13, kind=kind, seed=seed)).to("cuda")
        out = {"iris_mm": iris_diameter_mm, "workload": w13.name, "target": kind, "seed": seed,
               "optimiser": f"object space, step {beta:g}, momentum {mu:g}, {iters} iterations",
               "rays_in_resin_13": P13.info()["rays_in_resin"], "rays_total_13": P13.info()["n_rays"]}
        for name, P in (("chief_ray_model", P1), ("thirteen_ray_model", P13)):
            g = _optimise(P, f, iters, beta, mu)
            d = P13.forward_dose(g)
            out[name] = {"ver_in_13_ray_printer": P13.voxel_error_rate(d, f)[0]}
        return out
    finally:
        P13.close()
        P1.close()
