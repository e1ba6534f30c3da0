"""Fin-part simulation: the build-height comparison of Sec. 3 (Figs. 6 and 8) in the
non-telecentric printer of Sec. 2.6.1.  A part of n horizontal fins stacked above the
projector's optical axis is dosed (a) with Radon-method projections (Sec. 2.3) and (b)
with projections from the ray-traced optimiser, both simulated in the ray-traced printer;
a fin counts as formed when, at the binarisation threshold that minimises the voxel error
rate, at least `form` of its voxels cure and at least `form` of the gap above it stays
liquid.  The paper printed 9 fins (Radon: 3 formed, 3DRT: 9) and simulated 18 with 3DRT.
Every dose and projection comes from the CUDA library; this file holds masks and counts."""
from __future__ import annotations

import numpy as np
import torch

from . import inputs as I
from . import radon as R
from . import vamrt as V


def fin_masks(w: I.Workload, n_fins: int):
    """Boolean [nz][ny][nx] masks: per fin its slab inside the fin footprint, and the gap
    above it (between this fin and the next, or 1.25 mm above the last), spine excluded."""
    Z, Y, X = I.voxel_centres(w)
    hx = I.FIN_HALF_MM
    foot = (np.abs(X) <= hx) & (np.abs(Y) <= hx) & ~(Y >= hx - 1.0)       # footprint minus the spine
    fins, gaps = [], []
    for zb in I.fin_bottoms_mm(n_fins):
        zt = zb + I.FIN_THICK_MM
        fins.append(foot & (Z >= zb) & (Z <= zt))
        gaps.append(foot & (Z > zt) & (Z < zb + I.FIN_PERIOD_MM))
    return fins, gaps


def fins_formed(dose: torch.Tensor, w: I.Workload, n_fins: int, threshold_index: int, form: float = 0.9) -> dict:
    """Per fin, the cured fraction of the fin and the liquid fraction of the gap above it
    when voxels with floor(dose * 1024 / max(dose)) >= threshold_index cure."""
    d = dose.float()
    cured = torch.floor(d * (1024.0 / d.max())) >= threshold_index
    fins, gaps = fin_masks(w, n_fins)
    rows = []
    for fm, gm in zip(fins, gaps):
        fm_t = torch.from_numpy(fm).to(d.device)
        gm_t = torch.from_numpy(gm).to(d.device)
        c = float(cured[fm_t].float().mean()) if fm.any() else 0.0
        g = float((~cured[gm_t]).float().mean()) if gm.any() else 1.0
        rows.append({"fin_cured": c, "gap_liquid": g, "formed": bool(c >= form and g >= form)})
    return {"formed": sum(r["formed"] for r in rows), "of": n_fins, "per_fin": rows}


def fins_experiment(n_fins: int, iters: int | None = None, beta: float = 4.0, mu: float = 0.5) -> dict:
    """Radon-method projections vs the ray-traced optimiser (model step beta, momentum mu,
    `iters` iterations) on the n-fin part, both dosed by the ray-traced printer."""
    w = I.fins_workload(n_fins)
    iters = iters or w.osmo_iters
    P = V.Projector.from_workload(w, I.workload_pupil(w))
    wr = I.radon_workload(w)
    P_radon = V.Projector.from_workload(wr, I.workload_pupil(wr))
    try:
        f = torch.from_numpy(I.make_target(w)).to("cuda")
        model, prev = f.clone(), f.clone()
        proj = torch.empty(w.proj_shape, device=f.device)
        dose = torch.empty(w.vol_shape, device=f.device)
        for _ in range(iters):
            P.optimize(f, model=model, prev_model=prev, proj=proj, dose=dose, max_iter=1, tol=0.0, step=beta,
                       momentum=mu)
        ver_rt, idx_rt = P.voxel_error_rate(dose, f)
        g_r = R.radon_projections(P_radon, f, w.pixel_u_mm)
        d_r = P.forward_dose(g_r)
        ver_r, idx_r = P.voxel_error_rate(d_r, f)
        rt = fins_formed(dose, w, n_fins, idx_rt)
        rr = fins_formed(d_r, w, n_fins, idx_r)
        top = float(I.fin_bottoms_mm(n_fins)[-1]) + I.FIN_THICK_MM
        return {"workload": w.name, "fins": n_fins, "top_mm": top,
                "max_chief_ray_angle_deg_in_air": float(np.degrees(np.arctan(top / w.pupil_mm))),
                "ray_traced": {"optimiser": f"object space, step {beta:g}, momentum {mu:g}, {iters} iterations",
                               "ver": ver_rt, "fins_formed": rt["formed"], "per_fin": rt["per_fin"]},
                "radon": {"method": "Sec. 2.3 without the coordinate remap", "ver": ver_r,
                          "fins_formed": rr["formed"], "per_fin": rr["per_fin"]}}
    finally:
        P.close()
        P_radon.close()
