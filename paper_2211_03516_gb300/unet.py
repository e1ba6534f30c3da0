"""Learned warm start: a 3D U-Net whose convolutions run on the tensor cores through
the C ABI (vamrt_conv3d_bf16).  Activations are channels-last BF16 [D][H][W][C]."""
from __future__ import annotations

import ctypes

import torch

from . import vamrt as V


def _lib():
    L = V.lib()
    if not getattr(L, "_conv_ready", False):
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        L.vamrt_conv3d_bf16.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp]
        L.vamrt_conv3d_bf16.restype = ctypes.c_int
        L.vamrt_conv3d_tiling.argtypes = [i32, i32, i32, i32, i32, i32, vp]
        L.vamrt_conv3d_tiling.restype = ctypes.c_int
        L._conv_ready = True
    return L


_err_flags = {}


def _err_flag(device) -> torch.Tensor:
    key = str(device)
    if key not in _err_flags:
        _err_flags[key] = torch.zeros(1, dtype=torch.int32, device=device)
    return _err_flags[key]


def conv3d(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor | None = None, relu: bool = False,
           out_dtype=torch.bfloat16, out: torch.Tensor | None = None) -> torch.Tensor:
    """x [D][H][W][Cin] bf16, w [Cout][taps][Cin] bf16 (taps 27 or 1) -> y [D][H][W][Cout]."""
    if x.dtype != torch.bfloat16 or w.dtype != torch.bfloat16:
        raise TypeError("x and w must be bfloat16")
    if not (x.is_cuda and w.is_cuda and x.is_contiguous() and w.is_contiguous()):
        raise ValueError("x and w must be contiguous CUDA tensors")
    D, H, W, Cin = x.shape
    Cout, taps, Cin_w = w.shape
    if Cin_w != Cin:
        raise ValueError("channel mismatch")
    if out is None:
        out = torch.empty((D, H, W, Cout), device=x.device, dtype=out_dtype)
    b = bias.contiguous().float() if bias is not None else None
    err = _err_flag(x.device)
    st = _lib().vamrt_conv3d_bf16(x.data_ptr(), w.data_ptr(), b.data_ptr() if b is not None else None,
                                  out.data_ptr(), 1 if out.dtype == torch.float32 else 0, D, H, W, Cin, Cout, taps,
                                  1 if relu else 0, err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    V._check(st, "vamrt_conv3d_bf16")
    return out


def conv3d_tiling(D, H, W, cin, cout, taps):
    """(kernel, TZ, TY, Nt) that conv3d uses for this shape on the current device: kernel 1
    = halo-tile (regions of TZ planes x TY rows, Nt output channels per work item), 0 =
    the gather kernel."""
    out = (ctypes.c_int32 * 4)()
    V._check(_lib().vamrt_conv3d_tiling(D, H, W, cin, cout, taps, out), "vamrt_conv3d_tiling")
    return tuple(int(v) for v in out)


def check_errors(device="cuda:0"):
    """Raise if any tensor-core kernel reported a timed-out wait since the last check."""
    err = _err_flag(device)
    if int(err.item()) != 0:
        err.zero_()
        raise RuntimeError("a tensor-core kernel timed out waiting for its MMAs (output invalid)")


# ---------------------------------------------------------------------------------------
# thin wrappers of the remaining building blocks
# ---------------------------------------------------------------------------------------
def _ptr(t):
    return None if t is None else t.data_ptr()


def _s():
    return torch.cuda.current_stream().cuda_stream


def _setup_nn(L):
    if getattr(L, "_nn_ready", False):
        return L
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    L.vamrt_conv3d_wgrad_bf16.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, i32, vp, vp]
    L.vamrt_nn_resample.argtypes = [i32, vp, vp, i32, i32, i32, i32, vp]
    L.vamrt_nn_concat.argtypes = [vp, i32, vp, i32, vp, i64, i32, vp]
    L.vamrt_nn_relu_backward.argtypes = [vp, vp, i64, vp]
    L.vamrt_nn_bias_grad.argtypes = [vp, vp, i64, i32, vp]
    L.vamrt_nn_flip_weights.argtypes = [vp, vp, i32, i32, i32, vp]
    L.vamrt_nn_adam.argtypes = [vp, vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp]
    L.vamrt_nn_prepare_input.argtypes = [vp, vp, i32, i32, i32, i32, f32, vp]
    L.vamrt_nn_head_mse.argtypes = [vp, i32, vp, f32, vp, f32, vp, f32, vp, i32, i32, i32, i32, vp, vp]
    L.vamrt_nn_add.argtypes = [vp, vp, i64, vp]
    L.vamrt_projected_step.argtypes = [vp, vp, f32, i64, vp]
    L.vamrt_projected_adam.argtypes = [vp, vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp]
    L.vamrt_nn_absmax.argtypes = [vp, i64, vp, vp]
    for n in ("vamrt_conv3d_wgrad_bf16", "vamrt_nn_resample", "vamrt_nn_concat", "vamrt_nn_relu_backward",
              "vamrt_nn_bias_grad", "vamrt_nn_flip_weights", "vamrt_nn_adam", "vamrt_nn_prepare_input",
              "vamrt_nn_head_mse", "vamrt_nn_add", "vamrt_projected_step", "vamrt_projected_adam",
              "vamrt_nn_absmax"):
        getattr(L, n).restype = ctypes.c_int
    L._nn_ready = True
    return L


def _nn():
    return _setup_nn(_lib())


def conv3d_wgrad(x, dy, dw, taps):
    D, H, W, Cin = x.shape
    Cout = dy.shape[-1]
    V._check(_nn().vamrt_conv3d_wgrad_bf16(x.data_ptr(), dy.data_ptr(), dw.data_ptr(), D, H, W, Cin, Cout, taps,
                                           _err_flag(x.device).data_ptr(), _s()), "vamrt_conv3d_wgrad_bf16")


def avgpool2(x):
    D, H, W, C = x.shape
    out = torch.empty((D // 2, H // 2, W // 2, C), device=x.device, dtype=x.dtype)
    V._check(_nn().vamrt_nn_resample(0, x.data_ptr(), out.data_ptr(), D, H, W, C, _s()), "avgpool2")
    return out


def avgpool2_backward(g, fine_shape):
    D, H, W, C = fine_shape
    out = torch.empty(fine_shape, device=g.device, dtype=g.dtype)
    V._check(_nn().vamrt_nn_resample(1, g.data_ptr(), out.data_ptr(), D, H, W, C, _s()), "avgpool2_backward")
    return out


def upsample2(x):
    d, h, w, C = x.shape
    out = torch.empty((2 * d, 2 * h, 2 * w, C), device=x.device, dtype=x.dtype)
    V._check(_nn().vamrt_nn_resample(2, x.data_ptr(), out.data_ptr(), 2 * d, 2 * h, 2 * w, C, _s()), "upsample2")
    return out


def upsample2_backward(g):
    D, H, W, C = g.shape
    out = torch.empty((D // 2, H // 2, W // 2, C), device=g.device, dtype=g.dtype)
    V._check(_nn().vamrt_nn_resample(3, g.data_ptr(), out.data_ptr(), D, H, W, C, _s()), "upsample2_backward")
    return out


def concat(a, b):
    out = torch.empty(a.shape[:-1] + (a.shape[-1] + b.shape[-1],), device=a.device, dtype=a.dtype)
    npos = a.numel() // a.shape[-1]
    V._check(_nn().vamrt_nn_concat(a.data_ptr(), a.shape[-1], b.data_ptr(), b.shape[-1], out.data_ptr(), npos, 0,
                                   _s()), "concat")
    return out


def split(g, ca):
    cb = g.shape[-1] - ca
    a = torch.empty(g.shape[:-1] + (ca,), device=g.device, dtype=g.dtype)
    b = torch.empty(g.shape[:-1] + (cb,), device=g.device, dtype=g.dtype)
    npos = g.numel() // g.shape[-1]
    V._check(_nn().vamrt_nn_concat(a.data_ptr(), ca, b.data_ptr(), cb, g.data_ptr(), npos, 1, _s()), "split")
    return a, b


def absmax(x) -> torch.Tensor:
    """max |x| of an FP32 tensor, as a 1-element device tensor."""
    out = torch.empty(1, device=x.device, dtype=torch.float32)
    V._check(_nn().vamrt_nn_absmax(x.data_ptr(), x.numel(), out.data_ptr(), _s()), "absmax")
    return out


def add_(y, x):
    V._check(_nn().vamrt_nn_add(x.data_ptr(), y.data_ptr(), y.numel(), _s()), "add")
    return y


# ---------------------------------------------------------------------------------------
# the network
# ---------------------------------------------------------------------------------------
# (name, cin, cout, taps); every conv but the head is followed by ReLU
ARCH = [
    ("enc0a", 16, 16, 27), ("enc0b", 16, 16, 27),
    ("enc1a", 16, 32, 27), ("enc1b", 32, 32, 27),
    ("enc2a", 32, 64, 27), ("enc2b", 64, 64, 27),
    ("bota", 64, 128, 27), ("botb", 128, 128, 27),
    ("dec2a", 192, 64, 27), ("dec2b", 64, 64, 27),
    ("dec1a", 96, 32, 27), ("dec1b", 32, 32, 27),
    ("dec0a", 48, 16, 27), ("dec0b", 16, 16, 27),
    ("head", 16, 16, 1),
]


class Layer:
    def __init__(self, name, cin, cout, taps, device, rng):
        self.name, self.cin, self.cout, self.taps = name, cin, cout, taps
        std = (2.0 / (cin * taps)) ** 0.5
        w = (rng.standard_normal((cout, taps, cin)) * std).astype("float32")
        self.W = torch.from_numpy(w).to(device)                 # FP32 master
        self.b = torch.zeros(cout, device=device)
        self.Wb = self.W.to(torch.bfloat16)                     # BF16 copy for the kernels
        self.gW = torch.zeros_like(self.W)
        self.gb = torch.zeros_like(self.b)
        self.mW, self.vW = torch.zeros_like(self.W), torch.zeros_like(self.W)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)


class UNet3D:
    """4-level 3D U-Net (16/32/64/128 channels, two 3^3 convs per level, 2x average-pool
    down, nearest 2x up, skip concatenation, 1^3 head added to the input) over a projection stack
    [angles][v][u]; angles are padded circularly to a multiple of 8.  BF16 activations and
    weights, FP32 accumulation (tensor cores), FP32 master weights and Adam."""

    def __init__(self, device="cuda:0", seed=0):
        import numpy as np
        rng = np.random.default_rng(seed)
        self.device = torch.device(device)
        self.layers = {n: Layer(n, ci, co, t, self.device, rng) for (n, ci, co, t) in ARCH}
        self.step_count = 0
        self._acts = None

    # ---- forward ----
    def _conv(self, name, x, relu=True, out_f32=False):
        L = self.layers[name]
        return conv3d(x, L.Wb, L.b, relu=relu, out_dtype=torch.float32 if out_f32 else torch.bfloat16)

    def prepare(self, proj, scale, d_padded):
        A, Vv, U = proj.shape
        x = torch.empty((d_padded, Vv, U, 16), device=proj.device, dtype=torch.bfloat16)
        V._check(_nn().vamrt_nn_prepare_input(proj.data_ptr(), x.data_ptr(), A, Vv, U, d_padded, float(scale), _s()),
                 "prepare_input")
        return x

    def forward(self, x0):
        a = {"x0": x0}
        a["a0"] = self._conv("enc0a", x0)
        a["s0"] = self._conv("enc0b", a["a0"])
        a["p0"] = avgpool2(a["s0"])
        a["a1"] = self._conv("enc1a", a["p0"])
        a["s1"] = self._conv("enc1b", a["a1"])
        a["p1"] = avgpool2(a["s1"])
        a["a2"] = self._conv("enc2a", a["p1"])
        a["s2"] = self._conv("enc2b", a["a2"])
        a["p2"] = avgpool2(a["s2"])
        a["b1"] = self._conv("bota", a["p2"])
        a["b2"] = self._conv("botb", a["b1"])
        a["c2"] = concat(upsample2(a["b2"]), a["s2"])
        a["d2a"] = self._conv("dec2a", a["c2"])
        a["d2b"] = self._conv("dec2b", a["d2a"])
        a["c1"] = concat(upsample2(a["d2b"]), a["s1"])
        a["d1a"] = self._conv("dec1a", a["c1"])
        a["d1b"] = self._conv("dec1b", a["d1a"])
        a["c0"] = concat(upsample2(a["d1b"]), a["s0"])
        a["d0a"] = self._conv("dec0a", a["c0"])
        a["d0b"] = self._conv("dec0b", a["d0a"])
        a["z"] = self._conv("head", a["d0b"], relu=False, out_f32=True)
        self._acts = a
        return a["z"]

    def head(self, z, base, in_scale, target=None, want_grad=False, out_scale=1.0, target_scale=1.0):
        """Residual head: v = in_scale * base + z[...,0] on the first n_angles slices (base =
        the input projections).  Returns (out_scale * max(v, 0), loss, dz); loss = mean
        0.5 (v - target_scale * target)^2 when target is given."""
        Dp, Vv, Uu, cz = z.shape
        A = base.shape[0]
        out = torch.empty((A, Vv, Uu), device=z.device, dtype=torch.float32)
        loss = torch.zeros((), device=z.device, dtype=torch.float64) if target is not None else None
        dz = torch.empty((Dp, Vv, Uu, cz), device=z.device, dtype=torch.bfloat16) if want_grad else None
        V._check(_nn().vamrt_nn_head_mse(z.data_ptr(), cz, base.data_ptr(), float(in_scale), _ptr(target),
                                         float(target_scale), out.data_ptr(), float(out_scale), _ptr(dz), A, Vv, Uu,
                                         Dp, _ptr(loss), _s()), "head_mse")
        return out, loss, dz

    # ---- backward ----
    def _conv_bwd(self, name, x, y, dy, relu=True, need_dx=True):
        L = self.layers[name]
        if relu:
            V._check(_nn().vamrt_nn_relu_backward(y.data_ptr(), dy.data_ptr(), dy.numel(), _s()), "relu_backward")
        conv3d_wgrad(x, dy, L.gW, L.taps)
        npos = dy.numel() // dy.shape[-1]
        V._check(_nn().vamrt_nn_bias_grad(dy.data_ptr(), L.gb.data_ptr(), npos, L.cout, _s()), "bias_grad")
        if not need_dx:
            return None
        wt = torch.empty((L.cin, L.taps, L.cout), device=dy.device, dtype=torch.bfloat16)
        V._check(_nn().vamrt_nn_flip_weights(L.Wb.data_ptr(), wt.data_ptr(), L.cout, L.taps, L.cin, _s()), "flip")
        return conv3d(dy, wt, None, relu=False)

    def zero_grad(self):
        for L in self.layers.values():
            L.gW.zero_()
            L.gb.zero_()

    def backward(self, dz):
        a = self._acts
        g = self._conv_bwd("head", a["d0b"], None, dz, relu=False)
        g = self._conv_bwd("dec0b", a["d0a"], a["d0b"], g)
        g = self._conv_bwd("dec0a", a["c0"], a["d0a"], g)
        gu0, gs0 = split(g, a["c0"].shape[-1] - a["s0"].shape[-1])
        g = upsample2_backward(gu0)
        g = self._conv_bwd("dec1b", a["d1a"], a["d1b"], g)
        g = self._conv_bwd("dec1a", a["c1"], a["d1a"], g)
        gu1, gs1 = split(g, a["c1"].shape[-1] - a["s1"].shape[-1])
        g = upsample2_backward(gu1)
        g = self._conv_bwd("dec2b", a["d2a"], a["d2b"], g)
        g = self._conv_bwd("dec2a", a["c2"], a["d2a"], g)
        gu2, gs2 = split(g, a["c2"].shape[-1] - a["s2"].shape[-1])
        g = upsample2_backward(gu2)
        g = self._conv_bwd("botb", a["b1"], a["b2"], g)
        g = self._conv_bwd("bota", a["p2"], a["b1"], g)
        g = add_(avgpool2_backward(g, a["s2"].shape), gs2)
        g = self._conv_bwd("enc2b", a["a2"], a["s2"], g)
        g = self._conv_bwd("enc2a", a["p1"], a["a2"], g)
        g = add_(avgpool2_backward(g, a["s1"].shape), gs1)
        g = self._conv_bwd("enc1b", a["a1"], a["s1"], g)
        g = self._conv_bwd("enc1a", a["p0"], a["a1"], g)
        g = add_(avgpool2_backward(g, a["s0"].shape), gs0)
        g = self._conv_bwd("enc0b", a["a0"], a["s0"], g)
        self._conv_bwd("enc0a", a["x0"], a["a0"], g, need_dx=False)

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        L = _nn()
        for ly in self.layers.values():
            V._check(L.vamrt_nn_adam(ly.W.data_ptr(), ly.gW.data_ptr(), ly.mW.data_ptr(), ly.vW.data_ptr(),
                                     ly.Wb.data_ptr(), ly.W.numel(), lr, beta1, beta2, eps, self.step_count, _s()),
                     "adam")
            V._check(L.vamrt_nn_adam(ly.b.data_ptr(), ly.gb.data_ptr(), ly.mb.data_ptr(), ly.vb.data_ptr(), None,
                                     ly.b.numel(), lr, beta1, beta2, eps, self.step_count, _s()), "adam")

    LEVEL = {"enc0a": 0, "enc0b": 0, "enc1a": 1, "enc1b": 1, "enc2a": 2, "enc2b": 2, "bota": 3, "botb": 3,
             "dec2a": 2, "dec2b": 2, "dec1a": 1, "dec1b": 1, "dec0a": 0, "dec0b": 0, "head": 0}

    def forward_flops(self, d_padded, nv, nu):
        """Multiply-add FLOPs (2 per MAC) of the convolutions of one forward pass."""
        p0 = d_padded * nv * nu
        return sum(2.0 * (p0 / 8 ** self.LEVEL[n]) * L.cin * L.cout * L.taps for n, L in self.layers.items())

    def state_dict(self):
        return {n: (L.W.cpu(), L.b.cpu()) for n, L in self.layers.items()}

    def load_state_dict(self, sd):
        for n, (W, b) in sd.items():
            L = self.layers[n]
            L.W.copy_(W)
            L.b.copy_(b)
            L.Wb = L.W.to(torch.bfloat16)
