"""ctypes wrapper of the FP64 C oracle (vam_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check and by
the benchmark's CPU-baseline leg, never by the product path.  It imports nothing from
the CUDA package; workloads are passed in as any object with the attributes of a
workload (nx, ny, nz, voxel_mm, nu, nv, pixel_u_mm, ...).

Functions follow the paper section they implement:
  trace()          Sec. 2.1 ray generation and vector Snell refraction at the vial
  adjoint()        Sec. 2.4 projection (with Sec. 2.5's Fresnel/Beer-Lambert factors)
  adjoint_pixels() the same for single pixels (full-size sampled checks)
  forward()        Sec. 2.5 dose simulation
  sample_count()   samples per pass reaching the grid
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vam_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


class OrcGeom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("h", ctypes.c_double),
        ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
        ("pu", ctypes.c_double), ("pv", ctypes.c_double),
        ("pupil", ctypes.c_double), ("fnum", ctypes.c_double),
        ("m", ctypes.c_int32), ("pupil_xy", _dp),
        ("r_in", ctypes.c_double), ("wall", ctypes.c_double),
        ("n_out", ctypes.c_double), ("n_glass", ctypes.c_double), ("n_resin", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("n_angles", ctypes.c_int32), ("angles", _dp),
        ("step_vox", ctypes.c_double),
        ("unattenuated", ctypes.c_int32),
        ("n_surf", ctypes.c_int32), ("surf", _dp),
        ("obj_y", ctypes.c_double), ("mag", ctypes.c_double), ("aim", ctypes.c_double),
        ("aperture", ctypes.c_int32), ("per_pixel", ctypes.c_int32), ("seed", ctypes.c_uint64),
    ]


class OrcRay(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("k", ctypes.c_int32),
        ("origin", ctypes.c_double * 3), ("d0", ctypes.c_double * 3),
        ("p1", ctypes.c_double * 3), ("d1", ctypes.c_double * 3),
        ("e", ctypes.c_double * 3), ("d2", ctypes.c_double * 3),
        ("exit", ctypes.c_double * 3),
        ("ell", ctypes.c_double), ("t1", ctypes.c_double), ("t2", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, portable flags)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_trace.argtypes = [ctypes.POINTER(OrcGeom), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                ctypes.POINTER(OrcRay)]
        L.orc_trace.restype = ctypes.c_int
        L.orc_adjoint.argtypes = [ctypes.POINTER(OrcGeom), _dp, _dp]
        L.orc_adjoint.restype = None
        L.orc_forward.argtypes = [ctypes.POINTER(OrcGeom), _dp, _dp]
        L.orc_forward.restype = None
        L.orc_adjoint_pixel.argtypes = [ctypes.POINTER(OrcGeom), _dp, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32]
        L.orc_adjoint_pixel.restype = ctypes.c_double
        L.orc_sample_count.argtypes = [ctypes.POINTER(OrcGeom)]
        L.orc_sample_count.restype = ctypes.c_uint64
        L.orc_sizeof_geom.restype = ctypes.c_int32
        L.orc_lens_train.argtypes = [ctypes.POINTER(OrcGeom), _dp, _dp]
        L.orc_lens_train.restype = ctypes.c_int
        L.orc_sizeof_ray.restype = ctypes.c_int32
        L.orc_forward_pixel.argtypes = [ctypes.POINTER(OrcGeom), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
        L.orc_forward_pixel.restype = ctypes.c_int64
        L.orc_splitmix64.argtypes = [ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_jitter.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.orc_jitter.restype = ctypes.c_double
        L.orc_aperture_point.argtypes = [ctypes.POINTER(OrcGeom), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _dp]
        L.orc_aperture_point.restype = None
        assert L.orc_sizeof_geom() == ctypes.sizeof(OrcGeom)
        assert L.orc_sizeof_ray() == ctypes.sizeof(OrcRay)
        _lib = L
    return _lib


# aperture pattern names -> the oracle's own codes (see orc_geom.aperture)
_APERTURE = {"chief": 1, "stratified": 2, "sunflower": 3, "hex13": 4}


class _Geom:
    """Keeps the numpy arrays the C struct points to alive.  `pupil` is either an explicit
    (m, 2) list of stop points or a named pattern (an object with pattern, n_rays, seed and
    per_pixel attributes) that the oracle generates itself."""

    def __init__(self, w, pupil, angles, unattenuated=False):
        named = hasattr(pupil, "pattern")
        if named:
            m = int(pupil.n_rays)
            if pupil.pattern == "stratified":
                n = int(round(m ** 0.5))
                assert n * n == m, "stratified needs a square ray count"
            self.pupil_xy = np.zeros((m, 2))
        else:
            self.pupil_xy = np.ascontiguousarray(pupil, dtype=np.float64).reshape(-1, 2)
        self.angles = np.ascontiguousarray(angles, dtype=np.float64).ravel()
        g = OrcGeom()
        if named:
            g.aperture = _APERTURE[pupil.pattern]
            g.per_pixel = 1 if pupil.per_pixel else 0
            g.seed = int(pupil.seed) & 0xFFFFFFFFFFFFFFFF
        g.nx, g.ny, g.nz, g.h = w.nx, w.ny, w.nz, w.voxel_mm
        g.nu, g.nv, g.pu, g.pv = w.nu, w.nv, w.pixel_u_mm, w.pixel_v_mm
        g.pupil, g.fnum = w.pupil_mm, w.f_number
        g.m = self.pupil_xy.shape[0]
        g.pupil_xy = self.pupil_xy.ctypes.data_as(_dp)
        g.r_in, g.wall = w.r_inner_mm, w.wall_mm
        g.n_out, g.n_glass, g.n_resin = w.n_outside, w.n_glass, w.n_resin
        g.mu = w.mu_per_mm
        g.n_angles = self.angles.size
        g.angles = self.angles.ctypes.data_as(_dp)
        g.step_vox = w.step_vox
        g.unattenuated = 1 if unattenuated else 0
        lens = getattr(w, "lens", None)
        if lens is not None:
            self.surf = np.array([[sf.y_mm, sf.radius_mm, sf.n_after, sf.clear_mm, 1.0 if sf.stop else 0.0]
                                  for sf in lens.surfaces], dtype=np.float64).ravel()
            g.n_surf = len(lens.surfaces)
            g.surf = self.surf.ctypes.data_as(_dp)
            g.obj_y, g.mag, g.aim = lens.object_y_mm, lens.magnification, lens.aim_mm
        self.g = g

    @property
    def ref(self):
        return ctypes.byref(self.g)


def _angles_default(n):
    # theta_k = 2 pi k / N (Sec. 2.5: a full turn in equal steps)
    return 2.0 * np.pi * np.arange(n, dtype=np.float64) / n


def geom(w, pupil_xy, angles=None, unattenuated=False) -> _Geom:
    if angles is None:
        angles = _angles_default(w.n_angles)
    return _Geom(w, pupil_xy, angles, unattenuated)


def trace(w, pupil_xy, u, v, a) -> dict:
    """Sec. 2.1: one ray (pixel u, v; aperture sample a) through the vial at theta = 0."""
    G = geom(w, pupil_xy, np.zeros(1))
    r = OrcRay()
    lib().orc_trace(G.ref, u, v, a, ctypes.byref(r))
    out = {k: np.array(getattr(r, k)) for k in ("origin", "d0", "p1", "d1", "e", "d2", "exit")}
    out.update(status=r.status, k=r.k, ell=r.ell, t1=r.t1, t2=r.t2)
    return out


def adjoint(w, vol, pupil_xy, angles=None, unattenuated=False) -> np.ndarray:
    """Sec. 2.4 projection of a volume [nz][ny][nx] -> projections [n_angles][nv][nu] (FP64).
    unattenuated: the projection exactly as printed (no Fresnel / Beer-Lambert factors)."""
    G = geom(w, pupil_xy, angles, unattenuated)
    v = np.ascontiguousarray(vol, dtype=np.float64)
    assert v.shape == (w.nz, w.ny, w.nx)
    out = np.zeros((G.angles.size, w.nv, w.nu), dtype=np.float64)
    lib().orc_adjoint(G.ref, v.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def adjoint_pixels(w, vol, pupil_xy, pixels, angles=None) -> np.ndarray:
    """Projection values at the listed (k, v, u) pixels only."""
    G = geom(w, pupil_xy, angles)
    v = np.ascontiguousarray(vol, dtype=np.float64)
    L = lib()
    return np.array([L.orc_adjoint_pixel(G.ref, v.ctypes.data_as(_dp), int(k), int(vv), int(u))
                     for (k, vv, u) in pixels])


def forward(w, proj, pupil_xy, angles=None) -> np.ndarray:
    """Sec. 2.5 dose of projections [n_angles][nv][nu] -> dose [nz][ny][nx] (FP64)."""
    G = geom(w, pupil_xy, angles)
    p = np.ascontiguousarray(proj, dtype=np.float64)
    assert p.shape == (G.angles.size, w.nv, w.nu)
    out = np.zeros((w.nz, w.ny, w.nx), dtype=np.float64)
    lib().orc_forward(G.ref, p.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def forward_pixels(w, pupil, pixels, values, angles=None):
    """Sec. 2.5 dose of projections that are zero except at the listed (k, v, u) pixels
    (intensities `values`), as a sparse volume: (sorted flat voxel indices, dose there).
    Each pixel's contributions come from the same per-sample terms as forward(); the sums
    over pixels and samples are formed in FP64."""
    G = geom(w, pupil, angles)
    L = lib()
    idx_parts, val_parts = [], []
    cap = 1 << 16
    for (k, v, u), val in zip(pixels, values):
        while True:
            idx = np.empty(cap, np.int64)
            vv = np.empty(cap, np.float64)
            n = L.orc_forward_pixel(G.ref, int(k), int(v), int(u), float(val), idx.ctypes.data, vv.ctypes.data, cap)
            if n <= cap:
                break
            cap = int(n)
        idx_parts.append(idx[:n])
        val_parts.append(vv[:n])
    if not idx_parts:
        return np.zeros(0, np.int64), np.zeros(0)
    idx = np.concatenate(idx_parts)
    vals = np.concatenate(val_parts)
    uniq, inv = np.unique(idx, return_inverse=True)
    dose = np.zeros(uniq.size)
    np.add.at(dose, inv, vals)
    return uniq, dose


def lens_trace(w, origin, direction):
    """The oracle's lens-train stage alone: (ok, point on the last surface, direction
    behind it) for a ray (origin, unit direction) starting before the first surface."""
    G = geom(w, np.zeros((1, 2)), np.zeros(1))
    o = np.array(origin, dtype=np.float64)
    d = np.array(direction, dtype=np.float64)
    ok = lib().orc_lens_train(G.ref, o.ctypes.data_as(_dp), d.ctypes.data_as(_dp))
    return bool(ok), o, d


def aperture_points(w, pupil, u, v) -> np.ndarray:
    """Sec. 2.1 stop sampling: the (m, 2) stop points (xi, eta) of pixel (u, v)."""
    G = geom(w, pupil, np.zeros(1))
    out = np.zeros((G.g.m, 2))
    for a in range(G.g.m):
        lib().orc_aperture_point(G.ref, u, v, a, out[a].ctypes.data_as(_dp))
    return out


def jitter(seed, u, v, a, c) -> float:
    """The jitter number in [0, 1) of pixel (u, v), aperture sample a, component c."""
    return float(lib().orc_jitter(int(seed) & 0xFFFFFFFFFFFFFFFF, u, v, a, c))


def splitmix64(x) -> int:
    return int(lib().orc_splitmix64(int(x) & 0xFFFFFFFFFFFFFFFF))


def sample_count(w, pupil_xy, angles=None) -> int:
    G = geom(w, pupil_xy, angles)
    return int(lib().orc_sample_count(G.ref))
