"""The C-ABI library loads, exports what include/vamrt.h declares, and rejects bad
arguments on the host (no GPU needed, no compute call)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vamrt.h")


@pytest.fixture(scope="module")
def L():
    from paper_2211_03516_gb300 import build
    build.build()
    from paper_2211_03516_gb300 import vamrt
    return vamrt.lib()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vamrt_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for need in ("vamrt_make_projector", "vamrt_destroy_projector", "vamrt_adjoint", "vamrt_forward_dose",
                 "vamrt_optimize", "vamrt_sample_count", "vamrt_status_string"):
        assert need in syms


def test_library_exports_every_declared_symbol(L):
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_status_strings(L):
    L.vamrt_status_string.restype = ctypes.c_char_p
    assert L.vamrt_status_string(0) == b"ok"
    assert L.vamrt_status_string(1) == b"invalid argument"
    assert L.vamrt_status_string(99) == b"unknown status"


def _spec(**kw):
    from paper_2211_03516_gb300 import inputs as I
    from paper_2211_03516_gb300.vamrt import GeometrySpec
    w = I.TINY.scaled(**kw) if kw else I.TINY
    return GeometrySpec.from_workload(w, I.pupil_samples("chief", 1))


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 0, "grid extents"),
    ("nu", 0, "pixel array"),
    ("voxel_mm", -0.2, "voxel_mm"),
    ("voxel_mm", float("nan"), "voxel_mm"),
    ("r_inner_mm", 0.0, "r_inner_mm"),
    ("wall_mm", -1.0, "wall_mm"),
    ("n_glass", 0.0, "refractive"),
    ("mu_per_mm", -0.1, "mu_per_mm"),
    ("pupil_mm", 0.0, "pupil_mm"),
    ("f_number", -2.0, "f_number"),
    ("r_inner_mm", 7.0, "enclose"),
    ("step_vox", 100.0, "step_vox"),
])
def test_make_projector_rejects_bad_geometry(L, field, value, msg):
    from paper_2211_03516_gb300 import vamrt
    spec = _spec()
    setattr(spec, field, value)
    with pytest.raises(vamrt.VamrtError) as ei:
        vamrt.vamrt_make_projector(spec)
    assert ei.value.status == vamrt.VAMRT_EINVAL
    assert msg in str(ei.value)


def _lens(**changes):
    from dataclasses import replace
    from paper_2211_03516_gb300 import inputs as I
    L0 = I.telecentric_relay()
    surfs = list(L0.surfaces)
    for i, kw in changes.pop("surf", {}).items():
        surfs[i] = replace(surfs[i], **kw)
    return replace(L0, surfaces=tuple(surfs), **changes)


@pytest.mark.parametrize("lens,msg", [
    (dict(surf={1: dict(y_mm=-230.0)}), "increasing"),
    (dict(surf={2: dict(stop=False)}), "exactly one stop"),
    (dict(surf={2: dict(radius_mm=100.0)}), "stop must be a plane"),
    (dict(surf={0: dict(clear_mm=0.0)}), "clear_mm"),
    (dict(surf={4: dict(n_after=1.5)}), "outside medium"),
    (dict(object_y_mm=-100.0), "before the first surface"),
    (dict(magnification=0.0), "magnification"),
    (dict(aim_mm=-1.0), "aim_mm"),
])
def test_make_projector_rejects_bad_lens_train(L, lens, msg):
    """Lens-train geometry is checked on the host before anything runs on a device."""
    from paper_2211_03516_gb300 import vamrt
    spec = _spec()
    spec.lens = _lens(**lens)
    with pytest.raises(vamrt.VamrtError) as ei:
        vamrt.vamrt_make_projector(spec)
    assert ei.value.status == vamrt.VAMRT_EINVAL
    assert msg in str(ei.value)


def test_make_projector_rejects_pupil_outside_disk(L):
    from paper_2211_03516_gb300 import vamrt
    spec = _spec()
    spec.pupil = np.array([[0.9, 0.9]])
    with pytest.raises(vamrt.VamrtError, match="unit disk"):
        vamrt.vamrt_make_projector(spec)


@pytest.mark.parametrize("pattern,n,msg", [("stratified", 15, r"n\^2 rays"), ("hex13", 12, "13 rays"),
                                           ("chief", 2, "one ray")])
def test_make_projector_rejects_bad_aperture(L, pattern, n, msg):
    """Named aperture patterns are checked on the host: a stratified pattern needs a square
    ray count, the hexagonal filling 13 rays, the chief ray one."""
    from paper_2211_03516_gb300 import inputs as I
    from paper_2211_03516_gb300 import vamrt
    spec = _spec()
    spec.pupil = I.Aperture(pattern, n, seed=1, per_pixel=True)
    with pytest.raises(vamrt.VamrtError, match=msg):
        vamrt.vamrt_make_projector(spec)


def test_make_projector_rejects_unknown_aperture_code_and_flags(L):
    from paper_2211_03516_gb300 import vamrt
    for field, value, msg in (("aperture", 9, "unknown aperture pattern"), ("aperture_flags", 2, "aperture_flags")):
        g, keep = vamrt._to_struct(_spec())
        setattr(g, field, value)
        h = ctypes.c_void_p()
        assert L.vamrt_make_projector(ctypes.byref(g), None, ctypes.byref(h)) == vamrt.VAMRT_EINVAL
        L.vamrt_last_error.restype = ctypes.c_char_p
        assert msg in L.vamrt_last_error().decode()


def test_null_arguments_are_einval(L):
    from paper_2211_03516_gb300 import vamrt
    L.vamrt_last_error.restype = ctypes.c_char_p
    assert L.vamrt_adjoint(None, None, 0, None, 0, 0, None) == vamrt.VAMRT_EINVAL
    assert L.vamrt_forward_dose(None, None, 0, None, 0, 0, None) == vamrt.VAMRT_EINVAL
    assert L.vamrt_optimize(None, None, None, None, None, None, None, None) == vamrt.VAMRT_EINVAL
    assert L.vamrt_sample_count(None, None) == vamrt.VAMRT_EINVAL
    assert L.vamrt_make_projector(None, None, None) == vamrt.VAMRT_EINVAL
    L.vamrt_destroy_projector(None)  # no-op


def test_conv3d_weight_gradient_rejects_bad_arguments(L):
    """Host-side checks of vamrt_conv3d_wgrad_bf16 return EINVAL before any CUDA call (the
    addresses are never dereferenced)."""
    from paper_2211_03516_gb300 import vamrt
    f = L.vamrt_conv3d_wgrad_bf16
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32] * 6 + [ctypes.c_void_p] * 2
    good = dict(x=0x10000, dy=0x20000, dw=0x30000, d=2, h=3, w=16, cin=16, cout=16, taps=27, err=0x40000)
    cases = [dict(x=0x10008), dict(dy=0x20004), dict(x=None), dict(err=None), dict(w=24), dict(w=8),
             dict(cin=24), dict(cin=1040), dict(cout=272), dict(taps=9), dict(d=0),
             dict(d=1 << 14, h=1 << 13, w=16)]
    for bad in cases:
        a = {**good, **bad}
        st = f(a["x"], a["dy"], a["dw"], a["d"], a["h"], a["w"], a["cin"], a["cout"], a["taps"], a["err"], None)
        assert st == vamrt.VAMRT_EINVAL, bad


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2211_03516_gb300 import vamrt
    monkeypatch.setattr(vamrt, "_lib", None)
    monkeypatch.setattr(vamrt, "LIB_PATH", os.path.join(ROOT, "does-not-exist.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        vamrt.lib()
