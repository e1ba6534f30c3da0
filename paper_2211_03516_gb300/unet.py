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


def check_errors(device="cuda:0"):
    """Raise if any tensor-core kernel reported a timed-out wait since the last check."""
    err = _err_flag(device)
    if int(err.item()) != 0:
        err.zero_()
        raise RuntimeError("a tensor-core kernel timed out waiting for its MMAs (output invalid)")
