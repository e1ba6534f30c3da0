"""Optimiser and loss readings, in plain numpy (test infrastructure only).

Sec. 2.7 runs the object-space model optimisation (OSMO) of Rackson et al. with the
Radon transform and its inverse replaced by the ray-traced operators, and stops when the
absolute relative error between target and simulated dose falls below 0.5 %.  OSMO's
own equations are in that reference, not in the paper, so this file follows a stated
reading:

  m^0 = f_T
  g^k = max(0, P m^k)                 P: projection (the adjoint operator)
  d^k = A g^k                         A: dose operator
  dn^k = d^k / max_resin(d^k)         maximum over the resin voxels
  E^k = sum |dn^k - f_T| / sum f_T    the dose's L1 error relative to the target
  V^k = voxel error rate of dn^k      resin voxels misprinted at the best threshold
  m^{k+1} = max(0, m^k + (f_T - dn^k))
  stop after the update once V^k < tol, or after n_iter iterations.

"Absolute relative error" is read as V: the absolute mismatch between the target and
the dose as printed (thresholded), relative to the resin volume.  E cannot fall to
0.5 % for a binary target: a non-negative dose is never zero in the void along rays
that cross the part.

The thresholded dose loss (differentiable path; not in the paper):
  L(D) = mean_{v in P} relu(d_h - D_v)^2 + mean_{v in Q} relu(D_v - d_l)^2
with P = {f_T = 1}, Q = {f_T = 0}, and its gradient dL/dD.
"""
import numpy as np


def _resin(resin, shape):
    return np.ones(shape, dtype=bool) if resin is None else np.asarray(resin, dtype=bool)


def osmo(target, project, dose, n_iter, tol=0.005, beta=1.0, mu=0.0, m0=None, m_prev=None, resin=None,
         stop="ver"):
    """Returns (g, dn, m, errors E, voxel error rates V) after the iterations; project and
    dose are FP64 callables; resin is a boolean mask (default: every voxel).  beta scales
    the model update and mu adds heavy-ball momentum,
    m <- max(0, m + beta (f - dn) + mu (m - m_prev)); beta = 1, mu = 0 is the reading
    above, the others variants not in the paper.  m0 defaults to f, m_prev to m0 (at
    rest).  stop: "ver" (V < tol, the reading of Sec. 2.7) or "error" (E < tol)."""
    f = np.asarray(target, dtype=np.float64)
    rmask = _resin(resin, f.shape)
    fsum = f.sum()
    m = f.copy() if m0 is None else np.array(m0, dtype=np.float64)
    prev = m.copy() if m_prev is None else np.array(m_prev, dtype=np.float64)
    errors, vers = [], []
    g = dn = None
    for _ in range(n_iter):
        g = np.maximum(0.0, project(m))
        d = dose(g)
        dmax = d[rmask].max()
        if not dmax > 0.0:
            raise FloatingPointError("dose is zero everywhere in the resin")
        dn = d / dmax
        err = np.abs(dn - f).sum() / fsum
        errors.append(err)
        vers.append(voxel_error_rate(dn, f, rmask)[0])
        m, prev = np.maximum(0.0, m + beta * (f - dn) + mu * (m - prev)), m
        if (vers[-1] if stop == "ver" else err) < tol:
            break
    return g, dn, m, np.array(errors), np.array(vers)


def threshold_loss(dose, target, d_l, d_h):
    """(L, dL/dD) of the thresholded dose loss in FP64."""
    D = np.asarray(dose, dtype=np.float64)
    f = np.asarray(target)
    P = f > 0.5
    Q = ~P
    nP, nQ = max(int(P.sum()), 1), max(int(Q.sum()), 1)
    under = np.where(P, np.maximum(d_h - D, 0.0), 0.0)
    over = np.where(Q, np.maximum(D - d_l, 0.0), 0.0)
    L = (under ** 2).sum() / nP + (over ** 2).sum() / nQ
    grad = -2.0 * under / nP + 2.0 * over / nQ
    return L, grad


def voxel_error_rate(dose, target, resin_mask):
    """VER: fraction of resin voxels whose state at threshold tau_i = (i/1024) max(dose)
    differs from the target, minimised over i = 1..1023.  The above/below decision is
    the FP32 bin floor(dose * (1024 / max)) >= i (the dose's own precision); the counts
    are a direct sweep over thresholds (no histogram), independent of the CUDA path."""
    x = np.asarray(dose, dtype=np.float32)[resin_mask]
    f = np.asarray(target)[resin_mask] > 0.5
    m = np.float32(x.max())
    scale = np.float32(1024.0) / m if m > 0 else np.float32(0.0)
    b = np.clip(np.floor(x * scale), 0, 1023).astype(np.int64)
    best, best_i = None, 1
    for i in range(1, 1024):
        above = b >= i
        mis = int(np.count_nonzero(above != f))
        if best is None or mis < best:
            best, best_i = mis, i
    return best / x.size, best_i


def osmo_projections(target, g0, project, dose, n_iter, alpha=1.0, resin=None):
    """Projection-space iteration from g0 (reading; the learned warm start's continuation):
    d = A g; dn = d / max_resin(d); E = sum|dn - f| / sum f; g <- max(0, g + P(alpha (f - dn))).
    Without the model clamp this is the update OSMO makes to g = P m."""
    f = np.asarray(target, dtype=np.float64)
    rmask = _resin(resin, f.shape)
    fsum = f.sum()
    g = np.asarray(g0, dtype=np.float64).copy()
    errors = []
    dn = None
    for _ in range(n_iter):
        d = dose(g)
        dn = d / d[rmask].max()
        errors.append(np.abs(dn - f).sum() / fsum)
        g = np.maximum(0.0, g + project(alpha * (f - dn)))
    return g, dn, np.array(errors)


def threshold_adam(target, g0, project, dose, n_iter, step=0.8, d_l=0.8, d_h=1.0, b1=0.9, b2=0.999, eps=1e-12):
    """Adjoint-driven continuation from g0 >= 0 (reading; not in the paper): projected
    Adam steps on the thresholded dose loss, the gradient coming from the projection.
      g = g0 / mean_{v in P}(A g0)        the part's mean dose becomes 1 (the thresholds' scale)
      lr = step * mean_{g > 0}(g)
      iteration k = 1, 2, ...:
        D = A g;  L, G = threshold_loss(D);  grad = P G          P: projection (adjoint)
        m <- b1 m + (1 - b1) grad;  v <- b2 v + (1 - b2) grad^2
        g <- max(0, g - lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps))
    (Adam, Kingma and Ba: first-order steps scaled by bias-corrected moment estimates.)
    Returns (g after the last step, D of the last iteration, losses L per iteration)."""
    f = np.asarray(target, dtype=np.float64)
    g = np.asarray(g0, dtype=np.float64).copy()
    D = dose(g)
    g = g / D[f > 0.5].mean()
    lr = step * g[g > 0.0].mean()
    m = np.zeros_like(g)
    v = np.zeros_like(g)
    losses = []
    for k in range(1, n_iter + 1):
        D = dose(g)
        L, G = threshold_loss(D, f, d_l, d_h)
        losses.append(L)
        grad = project(G)
        m = b1 * m + (1.0 - b1) * grad
        v = b2 * v + (1.0 - b2) * grad * grad
        g = np.maximum(0.0, g - lr * (m / (1.0 - b1 ** k)) / (np.sqrt(v / (1.0 - b2 ** k)) + eps))
    return g, D, np.array(losses)


def export_u8(proj):
    """8-bit export (Sec. 2.7, reading: upper clip at mean + 3 sigma, projections >= 0):
    codes = round-half-even(255 min(max(g, 0), c) / c), c = mean + 3 sigma (population)."""
    g = np.asarray(proj, dtype=np.float64)
    c = g.mean() + 3.0 * g.std()
    codes = np.rint(255.0 * np.clip(g, 0.0, c) / c).astype(np.uint8)
    return codes, c
