"""Direct 3D convolution in FP64 (test infrastructure only): the warm-start network's
layer, y[p][co] = act(bias[co] + sum_{t, ci} x[p + off(t)][ci] w[co][t][ci]), stride 1,
zero padding, channels-last volumes [D][H][W][C], taps in (dz, dy, dx) order with dx
fastest.  Written as a plain sum over the 27 shifted copies of the input."""
import numpy as np


def tap_offsets(taps):
    if taps == 1:
        return [(0, 0, 0)]
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3d(x, w, bias=None, relu=False):
    """x [D][H][W][Cin], w [Cout][taps][Cin] -> y [D][H][W][Cout] (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    D, H, W, Cin = x.shape
    Cout, taps, _ = w.shape
    xp = np.zeros((D + 2, H + 2, W + 2, Cin))
    xp[1:-1, 1:-1, 1:-1] = x
    y = np.zeros((D, H, W, Cout))
    for t, (dz, dy, dx) in enumerate(tap_offsets(taps)):
        shifted = xp[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
        y += shifted @ w[:, t, :].T
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)
    if relu:
        y = np.maximum(y, 0.0)
    return y
