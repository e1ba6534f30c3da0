"""Radon-method baseline of Sec. 2.3, in plain numpy FP64 (test infrastructure only:
imported by the tests and the benchmark's checks, never by the product path).

Sec. 2.3 computes tomographic projections without ray tracing: the parallel-beam Radon
transform of every z-slice of the target, a Ram-Lak (ramp) filter applied to each
sinogram row, and negative values clipped to zero (light cannot be negative), followed
by a coordinate remap for refraction whose reference is not available here.

Reading of "a Ram-Lak filter in the Fourier domain": the band-limited ramp of filtered
backprojection on a detector of pitch tau, whose spatial kernel is
    h[0] = 1 / (4 tau^2),  h[n] = -1 / (pi^2 n^2 tau^2) for odd n,  h[n] = 0 for even n != 0,
applied as a linear (zero-padded) convolution, q[u] = tau * sum_n h[n] p[u - n] over the
row -- the product the Fourier-domain filter forms when the row is padded to at least
twice its length.  The Radon transform itself is the ray-traced projection with parallel
chief rays, no refraction and no attenuation (the index-matched, telecentric special case
of the projection operator), so this file holds only the filter.
"""
import numpy as np


def ramlak_taps(n):
    """h[k] * tau^2 for k = 0 .. n - 1 (the kernel is even: h[-k] = h[k])."""
    k = np.arange(n, dtype=np.float64)
    h = np.zeros(n, dtype=np.float64)
    h[0] = 0.25
    odd = k % 2 == 1
    h[odd] = -1.0 / (np.pi ** 2 * k[odd] ** 2)
    return h


def ramlak_filter(proj, tau, clamp=False):
    """Filter every row (last axis) of `proj`: q[u] = (1 / tau) sum_{u'} h_unit[u - u'] p[u'],
    with h_unit = tau^2 h; clamp: max(q, 0) afterwards (Sec. 2.3)."""
    p = np.asarray(proj, dtype=np.float64)
    nu = p.shape[-1]
    half = ramlak_taps(nu)
    kern = np.concatenate([half[:0:-1], half])          # taps -(nu-1) .. nu-1
    rows = p.reshape(-1, nu)
    out = np.empty_like(rows)
    for i, r in enumerate(rows):
        full = np.convolve(r, kern)                      # length 2 nu - 1 + nu - 1
        out[i] = full[nu - 1:2 * nu - 1] / tau
    if clamp:
        out = np.maximum(out, 0.0)
    return out.reshape(p.shape)
