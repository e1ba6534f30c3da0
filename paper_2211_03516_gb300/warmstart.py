"""Learned warm start for the projection optimiser.

The network (unet.UNet3D, tensor-core convolutions) maps a target's projections
A^T f -- the optimiser's own first projections -- to the projections the plain
optimiser reaches after many iterations.  Training pairs come from the plain ray-traced
optimiser itself (object-space iterations from m = f).  At inference the predicted
projections start an adjoint-driven continuation -- projected Adam steps on the thresholded
dose loss, gradients from the projection kernel (loss_curve) -- or the projection-space
iteration of vamrt_optimize, and the plain optimiser's voxel error rate (VER) judges the
result.  Both inputs and targets are
scaled by 1 / max(A^T f) so the network sees values in [0, 1].
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import inputs as I
from . import unet as U
from . import vamrt as V


def padded_angles(n_angles: int) -> int:
    return ((n_angles + 7) // 8) * 8


def _scale_of(y: torch.Tensor) -> float:
    m = float(U.absmax(y).item())
    return 1.0 / m if m > 0 else 1.0


def make_pairs(P: V.Projector, w, seeds, osmo_iters: int, device="cuda:0", kind="csg"):
    """[(f, A^T f, g*, scale)] on the device; g* = projections after osmo_iters plain iterations."""
    pairs = []
    for seed in seeds:
        f = torch.from_numpy(I.make_target(w, kind=kind, seed=int(seed))).to(device)
        if float(f.sum()) == 0.0:
            continue
        y = P.adjoint(f)
        res = P.optimize(f, max_iter=osmo_iters, tol=0.0)
        pairs.append((f, y, res["proj"], _scale_of(y)))
    return pairs


def train(net: U.UNet3D, pairs, epochs: int, lr: float = 1e-3, log=None):
    A = pairs[0][1].shape[0]
    Dp = padded_angles(A)
    losses = []
    for ep in range(epochs):
        tot = 0.0
        for i in np.random.default_rng(ep).permutation(len(pairs)):
            f, y, g, s = pairs[i]
            x0 = net.prepare(y, s, Dp)
            net.zero_grad()
            z = net.forward(x0)
            _, loss, dz = net.head(z, y, s, target=g, want_grad=True, target_scale=s)
            net.backward(dz)
            net.adam_step(lr)
            tot += float(loss.item())
        losses.append(tot / len(pairs))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.3e}")
    U.check_errors(net.device)
    return losses


def predict(net: U.UNet3D, y: torch.Tensor) -> torch.Tensor:
    """Warm-start projections from A^T f (same units as the optimiser's projections)."""
    A = y.shape[0]
    s = _scale_of(y)
    z = net.forward(net.prepare(y, s, padded_angles(A)))
    out, _, _ = net.head(z, y, s, out_scale=1.0 / s)
    return out


def ver_curve(P: V.Projector, f: torch.Tensor, iters: int, g0=None, dtype=torch.float32, step=0.5, beta=1.0,
              goal=None, mu=0.0):
    """VER after each iteration and cumulative device seconds: object space from m = f with
    model step beta and momentum mu when g0 is None, else projection space from g0 with
    relaxation step.  Stops early once VER <= goal when a goal is given."""
    vol = torch.empty_like(f)
    dose = torch.empty(f.shape, device=f.device, dtype=dtype)
    if g0 is None:
        model, proj, mode = f.clone(), torch.empty(P.proj_shape, device=f.device, dtype=dtype), "object"
    else:
        model, proj, mode = vol, g0.clone().to(dtype), "projections"
    prev = f.clone() if (g0 is None and mu) else None
    t, vers = 0.0, []
    times = []
    for _ in range(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.optimize(f, model=model, proj=proj, dose=dose, max_iter=1, tol=0.0, mode=mode,
                   step=beta if mode == "object" else step, momentum=mu if mode == "object" else 0.0,
                   prev_model=prev)
        e1.record()
        e1.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        times.append(t)
        vers.append(P.voxel_error_rate(dose, f)[0])
        if goal is not None and vers[-1] <= goal:
            break
    return np.array(vers), np.array(times)


def loss_curve(P: V.Projector, f: torch.Tensor, g0: torch.Tensor, iters: int, lr: float = 0.8, d_l: float = 0.8,
               d_h: float = 1.0, dtype=torch.bfloat16, goal=None):
    """Adjoint-driven continuation from g0: projected Adam steps on the thresholded dose
    loss L(D), D = A g, L = mean_P relu(d_h - D)^2 + mean_Q relu(D - d_l)^2 (the
    differentiable path: the gradient A^T dL/dD comes from the projection kernel).  g0 is
    first scaled so that the part's mean dose is 1; projections and dose are stored in
    `dtype` (FP32 master projections and moments); the Adam step is lr times the mean
    positive projection.  Returns (VER after each iteration, cumulative device seconds),
    stopping early once VER <= goal."""
    L = U._nn()
    n = P.proj_shape[0] * P.proj_shape[1] * P.proj_shape[2]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g = g0.float().clone()
    D = P.forward_dose(g.to(dtype), dose_dtype=dtype)
    g *= 1.0 / D.float()[f > 0.5].mean()
    gb = g.to(dtype)
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    grad = torch.empty_like(g)
    step = lr * float(g[g > 0].mean())
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    vers, times = [], []
    for k in range(iters):
        e0.record()
        P.forward_dose(gb, out=D)
        _, gD = P.threshold_loss(D, f, d_l, d_h, grad=True, grad_dtype=dtype)
        P.adjoint(gD, out=grad)
        V._check(L.vamrt_projected_adam(g.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), gb.data_ptr(), n,
                                        step, 0.9, 0.999, 1e-12, k + 1, V._stream(None)), "vamrt_projected_adam")
        vers.append(P.voxel_error_rate(D, f)[0])     # the stop check is part of the loop's time
        e1.record()
        e1.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        times.append(t)
        if goal is not None and vers[-1] <= goal:
            break
    return np.array(vers), np.array(times)


def compare(P: V.Projector, net: U.UNet3D, w, seeds, plain_iters: int, cont_iters: int, device="cuda:0", kind="csg",
            step=0.5, dtype=torch.float32, beta=4.0, mu=0.5, loss_iters=20, loss_lr=0.8, loss_dl=0.8):
    """Per held-out target: the plain FP32 run's final VER, and the iterations and device
    time to reach 1.01 x that VER for
      - the warm start (network inference, its time included) continued by the
        thresholded-loss Adam steps of loss_curve (BF16 storage), and the same continuation
        from g0 = max(0, A^T f) (no network);
      - the warm start continued by the projection-space iteration (relaxation `step`,
        storage dtype), and the same from g0 = max(0, A^T f);
      - the over-relaxed object-space loop (model step beta, momentum mu, from m = f,
        storage dtype), no network."""
    rows = []
    for seed in seeds:
        f = torch.from_numpy(I.make_target(w, kind=kind, seed=int(seed))).to(device)
        if float(f.sum()) == 0.0:
            continue
        v_plain, t_plain = ver_curve(P, f, plain_iters)
        goal = 1.01 * v_plain[-1]
        y = P.adjoint(f)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g_ws = predict(net, y)
        e1.record()
        e1.synchronize()
        t_inf = e0.elapsed_time(e1) / 1e3
        v_ws, t_ws = ver_curve(P, f, cont_iters, g0=g_ws, step=step, dtype=dtype)
        g_cold = P.adjoint(f, clamp_nonneg=True)
        v_cold, t_cold = ver_curve(P, f, cont_iters, g0=g_cold, step=step, dtype=dtype)
        v_rel, t_rel = ver_curve(P, f, plain_iters, dtype=dtype, beta=beta, goal=goal, mu=mu)
        v_wl, t_wl = loss_curve(P, f, g_ws, loss_iters, lr=loss_lr, d_l=loss_dl, goal=goal)
        v_cl, t_cl = loss_curve(P, f, g_cold, loss_iters, lr=loss_lr, d_l=loss_dl, goal=goal)

        def hit(v, t, extra=0.0):
            k = next((i for i, x in enumerate(v) if x <= goal), None)
            return (None, None) if k is None else (k + 1, float(t[k] + extra))

        k_ws, s_ws = hit(v_ws, t_ws, t_inf)
        k_cold, s_cold = hit(v_cold, t_cold)
        k_rel, s_rel = hit(v_rel, t_rel)
        k_wl, s_wl = hit(v_wl, t_wl, t_inf)
        k_cl, s_cl = hit(v_cl, t_cl)
        rows.append(dict(seed=int(seed), plain_final_ver=float(v_plain[-1]), plain_seconds=float(t_plain[-1]),
                         warm_loss_ver=v_wl.tolist(), warm_loss_iters_to_target=k_wl,
                         warm_loss_seconds_to_target=s_wl, cold_loss_ver=v_cl.tolist(),
                         cold_loss_iters_to_target=k_cl, cold_loss_seconds_to_target=s_cl,
                         warm_ver=v_ws.tolist(), cold_ver=v_cold.tolist(), plain_ver=v_plain.tolist(),
                         warm_iters_to_target=k_ws, warm_seconds_to_target=s_ws, inference_seconds=t_inf,
                         cold_iters_to_target=k_cold, cold_seconds_to_target=s_cold,
                         relaxed_iters_to_target=k_rel, relaxed_seconds_to_target=s_rel))
    return rows
