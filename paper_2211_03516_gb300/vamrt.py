"""Thin ctypes binding of the vamrt C ABI (include/vamrt.h).

Argument marshalling only: every numeric step runs in the CUDA library.  Tensors are
torch CUDA tensors (device memory and streams come from PyTorch); calls are queued on
the current torch stream.  If the compiled library is missing, every call raises: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvamrt.so")

VAMRT_OK, VAMRT_EINVAL, VAMRT_EUNSUPPORTED, VAMRT_ECUDA, VAMRT_ENOMEM, VAMRT_NOT_CONVERGED, VAMRT_NUMERIC = range(7)
VAMRT_F32, VAMRT_BF16, VAMRT_F16 = 0, 1, 2
VAMRT_ACCUMULATE, VAMRT_CLAMP_NONNEG, VAMRT_UNATTENUATED = 1, 2, 4
VAMRT_APERTURE = {"list": 0, "chief": 1, "stratified": 2, "sunflower": 3, "hex13": 4}
VAMRT_JITTER_PER_PIXEL = 1

_DTYPES = {torch.float32: VAMRT_F32, torch.bfloat16: VAMRT_BF16, torch.float16: VAMRT_F16}
_dp = ctypes.POINTER(ctypes.c_double)


class VamrtError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class Surface(ctypes.Structure):
    _fields_ = [("y_mm", ctypes.c_double), ("radius_mm", ctypes.c_double), ("n_after", ctypes.c_double),
                ("clear_mm", ctypes.c_double), ("is_stop", ctypes.c_int32)]


class Geometry(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("voxel_mm", ctypes.c_double),
        ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
        ("pixel_u_mm", ctypes.c_double), ("pixel_v_mm", ctypes.c_double),
        ("pupil_mm", ctypes.c_double), ("f_number", ctypes.c_double),
        ("rays_per_pixel", ctypes.c_int32), ("pupil_xy", _dp),
        ("r_inner_mm", ctypes.c_double), ("wall_mm", ctypes.c_double),
        ("n_outside", ctypes.c_double), ("n_glass", ctypes.c_double), ("n_resin", ctypes.c_double),
        ("mu_per_mm", ctypes.c_double),
        ("n_angles", ctypes.c_int32), ("angles_rad", _dp),
        ("step_vox", ctypes.c_double),
        ("n_surfaces", ctypes.c_int32), ("surfaces", ctypes.POINTER(Surface)),
        ("object_y_mm", ctypes.c_double), ("magnification", ctypes.c_double), ("aim_mm", ctypes.c_double),
        ("aperture", ctypes.c_int32), ("aperture_flags", ctypes.c_uint32), ("seed", ctypes.c_uint64),
    ]


class Info(ctypes.Structure):
    _fields_ = [("n_rays", ctypes.c_int64), ("rays_in_resin", ctypes.c_int64),
                ("samples_per_pass", ctypes.c_uint64), ("scratch_bytes", ctypes.c_uint64)]


class OptParams(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("check_every", ctypes.c_int32),
                ("proj_dtype", ctypes.c_int), ("dose_dtype", ctypes.c_int), ("timing", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("step", ctypes.c_double), ("momentum", ctypes.c_double),
                ("prev_model", ctypes.c_void_p), ("stop", ctypes.c_int32), ("d_l", ctypes.c_double),
                ("d_h", ctypes.c_double)]


class OptReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("final_error", ctypes.c_double), ("error_history", _dp),
                ("adjoint_ms", ctypes.c_double), ("forward_ms", ctypes.c_double), ("update_ms", ctypes.c_double),
                ("final_ver", ctypes.c_double), ("ver_history", _dp)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libvamrt.so (built in-tree by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first (no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
        L.vamrt_make_projector.argtypes = [ctypes.POINTER(Geometry), vp, ctypes.POINTER(vp)]
        L.vamrt_destroy_projector.argtypes = [vp]
        L.vamrt_destroy_projector.restype = None
        L.vamrt_get_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.vamrt_sample_count.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        L.vamrt_adjoint.argtypes = [vp, vp, i32, vp, i32, u32, vp]
        L.vamrt_forward_dose.argtypes = [vp, vp, i32, vp, i32, u32, vp]
        L.vamrt_optimize.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(OptParams), ctypes.POINTER(OptReport), vp]
        L.vamrt_copy_ray_table.argtypes = [vp, vp, vp, vp]
        L.vamrt_status_string.argtypes = [i32]
        L.vamrt_status_string.restype = ctypes.c_char_p
        L.vamrt_last_error.argtypes = []
        L.vamrt_last_error.restype = ctypes.c_char_p
        L.vamrt_threshold_loss.argtypes = [vp, vp, i32, vp, ctypes.c_double, ctypes.c_double, vp, vp, i32, vp]
        L.vamrt_threshold_loss.restype = i32
        L.vamrt_voxel_error_rate.argtypes = [vp, vp, i32, vp, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int32), vp]
        L.vamrt_voxel_error_rate.restype = i32
        L.vamrt_export_u8.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
        L.vamrt_export_u8.restype = i32
        L.vamrt_measure_smem_bandwidth.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
        L.vamrt_measure_smem_bandwidth.restype = i32
        L.vamrt_measure_l2_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
        L.vamrt_measure_l2_rates.restype = i32
        L.vamrt_ramlak_filter.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, u32, vp]
        L.vamrt_ramlak_filter.restype = i32
        L.vamrt_launch_count.argtypes = []
        L.vamrt_launch_count.restype = ctypes.c_uint64
        for name in ("vamrt_make_projector", "vamrt_get_info", "vamrt_sample_count", "vamrt_adjoint",
                     "vamrt_forward_dose", "vamrt_optimize", "vamrt_copy_ray_table"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(status: int, where: str, ok=(VAMRT_OK,)):
    if status not in ok:
        L = lib()
        detail = L.vamrt_last_error().decode() or L.vamrt_status_string(status).decode()
        raise VamrtError(status, where, detail)
    return status


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t: torch.Tensor, shape, name: str, dtypes=(torch.float32, torch.bfloat16, torch.float16)) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} dtype {t.dtype} not in {dtypes}")
    return t.data_ptr()


@dataclass
class GeometrySpec:
    """Host-side description mirrored into vamrt_geometry (see include/vamrt.h)."""
    nx: int
    ny: int
    nz: int
    voxel_mm: float
    nu: int
    nv: int
    pixel_u_mm: float
    pixel_v_mm: float
    pupil_mm: float
    f_number: float
    pupil: object                # a named aperture pattern (inputs.Aperture) or an explicit (m, 2) list
    r_inner_mm: float
    wall_mm: float
    n_outside: float
    n_glass: float
    n_resin: float
    mu_per_mm: float
    n_angles: int
    angles_rad: Optional[np.ndarray] = None
    step_vox: float = 0.5
    lens: object = None          # inputs.LensTrain or None (ideal pupil)

    @classmethod
    def from_workload(cls, w, pupil, angles_rad=None) -> "GeometrySpec":
        if not hasattr(pupil, "pattern"):
            pupil = np.asarray(pupil, dtype=np.float64).reshape(-1, 2)
        return cls(nx=w.nx, ny=w.ny, nz=w.nz, voxel_mm=w.voxel_mm, nu=w.nu, nv=w.nv,
                   pixel_u_mm=w.pixel_u_mm, pixel_v_mm=w.pixel_v_mm, pupil_mm=w.pupil_mm,
                   f_number=w.f_number, pupil=pupil,
                   r_inner_mm=w.r_inner_mm, wall_mm=w.wall_mm, n_outside=w.n_outside,
                   n_glass=w.n_glass, n_resin=w.n_resin, mu_per_mm=w.mu_per_mm,
                   n_angles=w.n_angles if angles_rad is None else len(angles_rad),
                   angles_rad=None if angles_rad is None else np.asarray(angles_rad, dtype=np.float64),
                   step_vox=w.step_vox, lens=getattr(w, "lens", None))


def _to_struct(spec: GeometrySpec):
    keep = []
    g = Geometry()
    for name, _ in Geometry._fields_:
        if name in ("pupil_xy", "angles_rad", "rays_per_pixel", "n_surfaces", "surfaces", "object_y_mm",
                    "magnification", "aim_mm", "aperture", "aperture_flags", "seed"):
            continue
        setattr(g, name, getattr(spec, name))
    if spec.lens is not None:
        surfs = (Surface * len(spec.lens.surfaces))(
            *[Surface(sf.y_mm, sf.radius_mm, sf.n_after, sf.clear_mm, 1 if sf.stop else 0) for sf in spec.lens.surfaces])
        keep.append(surfs)
        g.n_surfaces = len(spec.lens.surfaces)
        g.surfaces = ctypes.cast(surfs, ctypes.POINTER(Surface))
        g.object_y_mm = spec.lens.object_y_mm
        g.magnification = spec.lens.magnification
        g.aim_mm = spec.lens.aim_mm
    if hasattr(spec.pupil, "pattern"):
        g.aperture = VAMRT_APERTURE[spec.pupil.pattern]
        g.aperture_flags = VAMRT_JITTER_PER_PIXEL if spec.pupil.per_pixel else 0
        g.seed = int(spec.pupil.seed) & 0xFFFFFFFFFFFFFFFF
        g.rays_per_pixel = int(spec.pupil.n_rays)
        g.pupil_xy = None
    else:
        pupil = np.ascontiguousarray(spec.pupil, dtype=np.float64).reshape(-1, 2)
        keep.append(pupil)
        g.aperture = VAMRT_APERTURE["list"]
        g.rays_per_pixel = pupil.shape[0]
        g.pupil_xy = pupil.ctypes.data_as(_dp)
    if spec.angles_rad is not None:
        ang = np.ascontiguousarray(spec.angles_rad, dtype=np.float64)
        keep.append(ang)
        g.angles_rad = ang.ctypes.data_as(_dp)
    else:
        g.angles_rad = None
    return g, keep


def vamrt_make_projector(spec: GeometrySpec, stream=None) -> ctypes.c_void_p:
    g, keep = _to_struct(spec)
    h = ctypes.c_void_p()
    s = _stream(stream) if torch.cuda.is_available() else ctypes.c_void_p(0)
    _check(lib().vamrt_make_projector(ctypes.byref(g), s, ctypes.byref(h)), "vamrt_make_projector")
    del keep
    return h


class Projector:
    """Owns one vamrt_projector handle.  Operators run on the current torch stream."""

    def __init__(self, spec: GeometrySpec, stream=None):
        self.spec = spec
        self.handle = vamrt_make_projector(spec, stream)
        self.vol_shape = (spec.nz, spec.ny, spec.nx)
        self.proj_shape = (spec.n_angles, spec.nv, spec.nu)

    @classmethod
    def from_workload(cls, w, pupil, angles_rad=None, stream=None) -> "Projector":
        return cls(GeometrySpec.from_workload(w, pupil, angles_rad), stream)

    def close(self):
        if getattr(self, "handle", None):
            lib().vamrt_destroy_projector(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        i = Info()
        _check(lib().vamrt_get_info(self.handle, ctypes.byref(i)), "vamrt_get_info")
        return dict(n_rays=i.n_rays, rays_in_resin=i.rays_in_resin, samples_per_pass=i.samples_per_pass,
                    scratch_bytes=i.scratch_bytes)

    def sample_count(self) -> int:
        n = ctypes.c_uint64()
        _check(lib().vamrt_sample_count(self.handle, ctypes.byref(n)), "vamrt_sample_count")
        return int(n.value)

    def ray_table(self):
        n = self.info()["n_rays"]
        a4 = np.zeros((n, 4), np.float32)
        b4 = np.zeros((n, 4), np.float32)
        j2 = np.zeros((n, 2), np.int32)
        _check(lib().vamrt_copy_ray_table(self.handle, a4.ctypes.data, b4.ctypes.data, j2.ctypes.data),
               "vamrt_copy_ray_table")
        return a4, b4, j2

    def adjoint(self, vol: torch.Tensor, out: Optional[torch.Tensor] = None, proj_dtype=torch.float32,
                accumulate=False, clamp_nonneg=False, unattenuated=False, stream=None) -> torch.Tensor:
        """A^T: volume [nz][ny][nx] -> projections [n_angles][nv][nu] (vamrt_adjoint).
        unattenuated: the paper-literal projection (no Fresnel / Beer-Lambert factors)."""
        if out is None:
            out = torch.empty(self.proj_shape, device=vol.device, dtype=proj_dtype)
        vp = _dev_ptr(vol, self.vol_shape, "vol")
        pp = _dev_ptr(out, self.proj_shape, "proj")
        flags = ((VAMRT_ACCUMULATE if accumulate else 0) | (VAMRT_CLAMP_NONNEG if clamp_nonneg else 0)
                 | (VAMRT_UNATTENUATED if unattenuated else 0))
        _check(lib().vamrt_adjoint(self.handle, vp, _DTYPES[vol.dtype], pp, _DTYPES[out.dtype], flags,
                                   _stream(stream)), "vamrt_adjoint")
        return out

    def forward_dose(self, proj: torch.Tensor, out: Optional[torch.Tensor] = None, dose_dtype=torch.float32,
                     accumulate=False, stream=None) -> torch.Tensor:
        """A: projections [n_angles][nv][nu] -> dose [nz][ny][nx] (vamrt_forward_dose)."""
        if out is None:
            out = torch.empty(self.vol_shape, device=proj.device, dtype=dose_dtype)
        pp = _dev_ptr(proj, self.proj_shape, "proj")
        dp = _dev_ptr(out, self.vol_shape, "dose")
        flags = VAMRT_ACCUMULATE if accumulate else 0
        _check(lib().vamrt_forward_dose(self.handle, pp, _DTYPES[proj.dtype], dp, _DTYPES[out.dtype], flags,
                                        _stream(stream)), "vamrt_forward_dose")
        return out

    def threshold_loss(self, dose: torch.Tensor, target: torch.Tensor, d_l: float, d_h: float, grad=True,
                       grad_dtype=torch.float32, stream=None):
        """(L as a 0-d float64 CUDA tensor, dL/dD or None) (vamrt_threshold_loss)."""
        loss = torch.empty((), device=dose.device, dtype=torch.float64)
        dp = _dev_ptr(dose, self.vol_shape, "dose")
        tp = _dev_ptr(target, self.vol_shape, "target", (torch.float32,))
        g = torch.empty(self.vol_shape, device=dose.device, dtype=grad_dtype) if grad else None
        _check(lib().vamrt_threshold_loss(self.handle, dp, _DTYPES[dose.dtype], tp, float(d_l), float(d_h),
                                          loss.data_ptr(), g.data_ptr() if g is not None else None,
                                          _DTYPES[grad_dtype], _stream(stream)), "vamrt_threshold_loss")
        return loss, g

    def voxel_error_rate(self, dose: torch.Tensor, target: torch.Tensor, stream=None):
        """(VER, best threshold index) of a dose against the binary target (vamrt_voxel_error_rate)."""
        ver = ctypes.c_double()
        idx = ctypes.c_int32()
        _check(lib().vamrt_voxel_error_rate(self.handle, _dev_ptr(dose, self.vol_shape, "dose"), _DTYPES[dose.dtype],
                                            _dev_ptr(target, self.vol_shape, "target", (torch.float32,)),
                                            ctypes.byref(ver), ctypes.byref(idx), _stream(stream)),
               "vamrt_voxel_error_rate")
        return float(ver.value), int(idx.value)

    def export_u8(self, proj: torch.Tensor, stream=None):
        """(uint8 codes, dequantised f32 projections, clip value c) (vamrt_export_u8)."""
        pp = _dev_ptr(proj, self.proj_shape, "proj")
        codes = torch.empty(self.proj_shape, device=proj.device, dtype=torch.uint8)
        deq = torch.empty(self.proj_shape, device=proj.device, dtype=torch.float32)
        clip = ctypes.c_double()
        _check(lib().vamrt_export_u8(self.handle, pp, _DTYPES[proj.dtype], codes.data_ptr(), deq.data_ptr(),
                                     ctypes.byref(clip), _stream(stream)), "vamrt_export_u8")
        return codes, deq, float(clip.value)

    def optimize(self, target: torch.Tensor, model: Optional[torch.Tensor] = None, max_iter=10, tol=0.005,
                 check_every=1, proj_dtype=torch.float32, dose_dtype=torch.float32, proj=None, dose=None,
                 timing=False, mode="object", step=1.0, momentum=0.0, prev_model=None, stop="ver",
                 d_l=0.0, d_h=0.0, stream=None) -> dict:
        """Projection optimisation (vamrt_optimize).  Returns g, dn, model, errors, converged.
        mode "object": OSMO on the model (model in = m0, default the target), model step
        `step` (1 = the plain update) and heavy-ball `momentum` (0 = none), whose previous
        model lives in prev_model (in: the model before m0 -- a copy of m0 to start at rest,
        made here when prev_model is None; out: updated; pass the same buffer back to keep
        momentum across calls);
        mode "projections": iterate on proj (in = g0, required), model = workspace;
        mode "gradient": projected Adam steps on the thresholded dose loss (thresholds d_l,
        d_h; both 0 = 0.8, 1.0) from proj (in = g0, required; Adam step `step` x the mean
        projection, 0 = 0.8), model = volume workspace, `errors` = the loss per iteration.
        stop: "ver" (the voxel error rate V < tol, the reading of Sec. 2.7's stop) or
        "error" (E < tol); `vers` holds V of the checked iterations."""
        modes = {"object": 0, "projections": 1, "gradient": 2}
        if mode not in modes:
            raise ValueError("mode must be 'object', 'projections' or 'gradient'")
        if mode != "object" and proj is None:
            raise ValueError(f"{mode} mode needs the starting projections in proj")
        if model is None:
            model = target.clone() if mode == "object" else torch.empty_like(target)
        if momentum and prev_model is None:
            prev_model = model.clone()
        pm = _dev_ptr(prev_model, self.vol_shape, "prev_model", (torch.float32,)) if momentum else None
        if proj is None:
            proj = torch.empty(self.proj_shape, device=target.device, dtype=proj_dtype)
        if dose is None:
            dose = torch.empty(self.vol_shape, device=target.device, dtype=dose_dtype)
        tp = _dev_ptr(target, self.vol_shape, "target", (torch.float32,))
        mp = _dev_ptr(model, self.vol_shape, "model", (torch.float32,))
        pp = _dev_ptr(proj, self.proj_shape, "proj")
        dp = _dev_ptr(dose, self.vol_shape, "dose")
        params = OptParams(max_iter=max_iter, tol=tol, check_every=check_every, proj_dtype=_DTYPES[proj.dtype],
                           dose_dtype=_DTYPES[dose.dtype], timing=1 if timing else 0,
                           mode=modes[mode], step=float(step), momentum=float(momentum),
                           prev_model=pm, stop={"ver": 0, "error": 1}[stop], d_l=float(d_l), d_h=float(d_h))
        hist = np.zeros(max_iter, dtype=np.float64)
        vhist = np.full(max_iter, np.nan)
        rep = OptReport(iterations=0, final_error=math.nan, error_history=hist.ctypes.data_as(_dp),
                        final_ver=math.nan, ver_history=vhist.ctypes.data_as(_dp))
        st = _check(lib().vamrt_optimize(self.handle, tp, mp, pp, dp, ctypes.byref(params), ctypes.byref(rep),
                                         _stream(stream)), "vamrt_optimize", ok=(VAMRT_OK, VAMRT_NOT_CONVERGED))
        return dict(proj=proj, dose=dose, model=model, prev_model=prev_model, errors=hist[:rep.iterations].copy(),
                    vers=vhist[:rep.iterations].copy(), final_ver=rep.final_ver,
                    iterations=rep.iterations, final_error=rep.final_error, converged=(st == VAMRT_OK),
                    adjoint_ms=rep.adjoint_ms, forward_ms=rep.forward_ms, update_ms=rep.update_ms)


def ramlak_filter(proj: torch.Tensor, pixel_mm: float, clamp: bool = False, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    """Ram-Lak filter along the last axis of an f32 CUDA tensor (vamrt_ramlak_filter, the
    Radon-method baseline of Sec. 2.3); clamp clips negatives to zero; out may be proj."""
    if not isinstance(proj, torch.Tensor) or not proj.is_cuda or proj.dtype != torch.float32:
        raise TypeError("proj must be a float32 CUDA tensor")
    if not proj.is_contiguous():
        raise ValueError("proj must be contiguous")
    if out is None:
        out = torch.empty_like(proj)
    if out.shape != proj.shape or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor of proj's shape")
    nu = proj.shape[-1]
    rows = proj.numel() // nu if nu else 0
    _check(lib().vamrt_ramlak_filter(proj.data_ptr(), out.data_ptr(), rows, nu, float(pixel_mm),
                                     VAMRT_CLAMP_NONNEG if clamp else 0, _stream(stream)), "vamrt_ramlak_filter")
    return out


def vamrt_measure_smem_bandwidth(stream=None) -> float:
    """Measured shared-memory read bandwidth of the current GPU, bytes/s."""
    out = ctypes.c_double()
    _check(lib().vamrt_measure_smem_bandwidth(ctypes.byref(out), _stream(stream)), "vamrt_measure_smem_bandwidth")
    return float(out.value)


def vamrt_measure_l2_rates(stream=None):
    """(L2 read bandwidth in bytes/s, L2 16-byte vector reductions per s) of the current GPU."""
    rd, red = ctypes.c_double(), ctypes.c_double()
    _check(lib().vamrt_measure_l2_rates(ctypes.byref(rd), ctypes.byref(red), _stream(stream)),
           "vamrt_measure_l2_rates")
    return float(rd.value), float(red.value)


def vamrt_launch_count() -> int:
    """Kernels the library has launched in this process."""
    return int(lib().vamrt_launch_count())


def vamrt_adjoint(p: Projector, vol, out=None, **kw):
    return p.adjoint(vol, out, **kw)


def vamrt_forward_dose(p: Projector, proj, out=None, **kw):
    return p.forward_dose(proj, out, **kw)


def vamrt_optimize(p: Projector, target, **kw):
    return p.optimize(target, **kw)


def vamrt_sample_count(p: Projector) -> int:
    return p.sample_count()
