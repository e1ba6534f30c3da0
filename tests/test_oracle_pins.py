"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: closed forms in the
limits where the method reduces to a textbook result (parallel-beam Radon chords,
linear fields, Beer-Lambert sums), the invariants of Snell's law across coaxial
cylinders, the textbook angle form of the Fresnel equations, the transpose relation
between the projection and dose operators, a fine-step integration with a library
interpolator, and numbers printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from oracle import optics as OP
from oracle import osmo as OS
from oracle import vam_oracle as O
from paper_2211_03516_gb300 import inputs as I
from paper_2211_03516_gb300.inputs import INF, Workload, default_angles, pupil_samples, voxel_centres

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_w(**kw):
    base = dict(name="pin", nx=24, ny=24, nz=24, voxel_mm=0.5, nu=21, nv=7, pixel_u_mm=0.55,
                pixel_v_mm=0.5, n_angles=7, pupil_mm=INF, f_number=INF, pupil_pattern="chief",
                rays_per_pixel=1, r_inner_mm=5.0, wall_mm=1.0, n_outside=1.0, n_glass=1.0,
                n_resin=1.0, mu_per_mm=0.0, step_vox=0.5)
    base.update(kw)
    return Workload(**base)


def refracting_w(**kw):
    base = dict(pupil_mm=60.0, f_number=3.0, pupil_pattern="sunflower", rays_per_pixel=5,
                n_glass=1.47, n_resin=1.50, mu_per_mm=0.15)
    base.update(kw)
    return small_w(**base)


def pixel_x(w):
    return (np.arange(w.nu) - (w.nu - 1) / 2.0) * w.pixel_u_mm


def pixel_z(w):
    return (np.arange(w.nv) - (w.nv - 1) / 2.0) * w.pixel_v_mm


CHIEF = pupil_samples("chief", 1)


# --- a1-a4: parallel-beam (Radon) limit ------------------------------------------------
def test_radon_limit_chord_lengths():
    """Telecentric, zero etendue, index matched, mu = 0, unit field: y = 2 sqrt(R^2 - b^2)."""
    w = small_w()
    y = O.adjoint(w, np.ones(w.vol_shape), CHIEF)
    xu = pixel_x(w)
    R = w.r_inner_mm
    chord = np.where(np.abs(xu) < R, 2.0 * np.sqrt(np.maximum(R * R - xu * xu, 0.0)), 0.0)
    assert (chord == 0).sum() == 2  # the two outer columns only cross the glass wall
    np.testing.assert_allclose(y, np.broadcast_to(chord, y.shape), rtol=1e-12, atol=1e-12)


def test_linear_field_fixes_rotation_axes_and_centre():
    """Trilinear weights reproduce a linear field exactly and the midpoint rule integrates
    it exactly, so each pixel equals chord x field(segment midpoint).  The midpoint of the
    pixel's chord at angle theta sits at R(theta)(x_u, 0, z_v): this fixes the rotation
    sense, the axis order and the voxel-centre convention."""
    w = small_w(n_angles=9)
    Z, Y, X = voxel_centres(w)
    al, be, ga, ze = 0.7, 0.31, -0.23, 0.17
    V = al + be * X + ga * Y + ze * Z
    y = O.adjoint(w, V, CHIEF)
    th = default_angles(w.n_angles)[:, None, None]
    xu = pixel_x(w)[None, None, :]
    zv = pixel_z(w)[None, :, None]
    R = w.r_inner_mm
    chord = np.where(np.abs(xu) < R, 2.0 * np.sqrt(np.maximum(R * R - xu * xu, 0.0)), 0.0)
    expect = chord * (al + be * np.cos(th) * xu + ga * np.sin(th) * xu + ze * zv)
    np.testing.assert_allclose(y, expect, rtol=1e-11, atol=1e-11)


def test_beer_lambert_sum_closed_form_and_midpoint_bound():
    """Unit field, mu > 0: sum_j delta exp(-mu (j+1/2) delta) is a geometric series, and
    it lies within the midpoint-rule bound mu^2 delta^2 ell / 24 of (1 - exp(-mu ell))/mu."""
    mu = 0.35
    w = small_w(mu_per_mm=mu)
    y = O.adjoint(w, np.ones(w.vol_shape), CHIEF)
    R, ds = w.r_inner_mm, w.step_vox * w.voxel_mm
    for u, x in enumerate(pixel_x(w)):
        if abs(x) >= R:
            assert np.all(y[:, :, u] == 0.0)
            continue
        ell = 2.0 * math.sqrt(R * R - x * x)
        K = math.ceil(ell / ds - 1e-9)
        dl = ell / K
        geo = dl * math.exp(-mu * dl / 2) * (1 - math.exp(-mu * ell)) / (1 - math.exp(-mu * dl))
        np.testing.assert_allclose(y[:, :, u], geo, rtol=1e-12)
        exact = (1 - math.exp(-mu * ell)) / mu
        assert abs(y[0, 0, u] - exact) <= mu * mu * dl * dl * ell / 24 * (1 + 1e-9)


def test_sample_count_closed_form_with_z_clip():
    """Telecentric chief rays stay at height z_v; rows whose footprint misses the grid
    (q_z outside (-1, nz)) add no samples; the others add K = ceil(ell/ds) each."""
    w = small_w(nv=40, n_angles=5)
    ds = w.step_vox * w.voxel_mm
    R = w.r_inner_mm
    per_row = sum(math.ceil(2 * math.sqrt(R * R - x * x) / ds - 1e-9) for x in pixel_x(w) if abs(x) < R)
    qz = pixel_z(w) / w.voxel_mm + (w.nz - 1) / 2.0
    rows = int(np.sum((qz > -1) & (qz < w.nz)))
    assert 0 < rows < w.nv
    assert O.sample_count(w, CHIEF) == w.n_angles * rows * per_row


# --- a1: ray generator ------------------------------------------------------------------
def test_ray_generator_definition_non_telecentric():
    w = refracting_w()
    P = pupil_samples("disk", 5, seed=3)
    D = w.pupil_mm / w.f_number
    for (u, v, a) in [(0, 0, 0), (10, 3, 2), (20, 6, 4), (7, 1, 1)]:
        r = O.trace(w, P, u, v, a)
        C = np.array([P[a, 0] * D / 2, -w.pupil_mm, P[a, 1] * D / 2])
        Q = np.array([pixel_x(w)[u], 0.0, pixel_z(w)[v]])
        np.testing.assert_allclose(r["origin"], C, atol=1e-14)
        np.testing.assert_allclose(r["d0"], (Q - C) / np.linalg.norm(Q - C), atol=1e-15)


# --- a1: aperture-stop sampling (Sec. 2.1; patterns of the workloads) --------------------
def test_splitmix64_reference_output():
    """splitmix64 from state 0 gives 0xE220A8397B1DCDAF, the first output of the published
    generator seeded with 0; the jitter number is its top 53 bits scaled by 2^-53."""
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    assert O.jitter(0, 0, 0, 0, 0) == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53


def test_jitter_numbers_are_uniform_and_keyed_by_every_index():
    """Chi-square of 20000 jitter numbers over 20 bins stays in the bulk of its distribution
    (19 degrees of freedom), and changing any one of u, v, a, c or the seed changes it."""
    vals = np.array([O.jitter(7, u, v, a, c) for u in range(25) for v in range(20) for a in range(20) for c in (0, 1)])
    assert vals.min() >= 0.0 and vals.max() < 1.0
    counts = np.histogram(vals, bins=20, range=(0.0, 1.0))[0]
    exp = vals.size / 20
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 43.8                      # 99.9th percentile of chi-square(19)
    base = O.jitter(7, 3, 4, 5, 0)
    for args in ((8, 3, 4, 5, 0), (7, 4, 4, 5, 0), (7, 3, 5, 5, 0), (7, 3, 4, 6, 0), (7, 3, 4, 5, 1)):
        assert O.jitter(*args) != base


def _uncentric(x, y):
    """Inverse of the concentric square-to-disk map: the point of [-1,1]^2 that maps to
    (x, y) (written from the map's definition: a square ring of half-width r goes to the
    circle of radius r, its four sides to the four quarter-circles centred on the axes)."""
    r = math.hypot(x, y)
    phi = math.atan2(y, x)
    if phi < -math.pi / 4:
        phi += 2 * math.pi
    if phi <= math.pi / 4:                   # right side: p = r, phi = (pi/4) q / p
        return r, 4 * phi * r / math.pi
    if phi <= 3 * math.pi / 4:               # top: q = r, phi = pi/2 - (pi/4) p / q
        return (math.pi / 2 - phi) * 4 * r / math.pi, r
    if phi <= 5 * math.pi / 4:               # left: p = -r, phi - pi = (pi/4) q / p
        return -r, -4 * (phi - math.pi) * r / math.pi
    return (phi - 3 * math.pi / 2) * 4 * r / math.pi, -r    # bottom: q = -r


def test_stratified_pattern_one_point_per_stratum():
    """n x n stratified jitter: ray a = i n + k of every pixel lies in the unit disk and maps
    back (inverse concentric map) into stratum (i, k) of [-1,1]^2; per-pixel jitter gives
    different points to different pixels, shared jitter the same ones."""
    w = small_w(pupil_mm=60.0, f_number=3.0, pupil_pattern="stratified4x4", rays_per_pixel=16)
    ap = I.workload_pupil(w)
    assert ap.per_pixel
    n = 4
    for (u, v) in [(0, 0), (5, 2), (20, 6)]:
        pts = O.aperture_points(w, ap, u, v)
        assert np.all(np.hypot(pts[:, 0], pts[:, 1]) <= 1.0)
        for a, (x, y) in enumerate(pts):
            p, q = _uncentric(x, y)
            assert (int((p + 1) * n / 2), int((q + 1) * n / 2)) == (a // n, a % n)
    assert not np.array_equal(O.aperture_points(w, ap, 0, 0), O.aperture_points(w, ap, 1, 0))
    shared = I.Aperture("stratified", 16, seed=0, per_pixel=False)
    np.testing.assert_array_equal(O.aperture_points(w, shared, 0, 0), O.aperture_points(w, shared, 9, 3))


def test_stratified_pattern_is_uniform_over_the_disk():
    """The concentric map preserves area fractions, so jittered strata fill the disk
    uniformly: over 400 pixels x 16 rays the fraction inside r = 1/2 is 1/4 and inside the
    quarter x > 0, y > 0 is 1/4 (within a few binomial standard deviations)."""
    w = small_w(nu=20, nv=20, pupil_mm=60.0, f_number=3.0, pupil_pattern="stratified4x4", rays_per_pixel=16)
    ap = I.workload_pupil(w)
    pts = np.concatenate([O.aperture_points(w, ap, u, v) for u in range(20) for v in range(20)])
    inner = np.mean(np.hypot(pts[:, 0], pts[:, 1]) < 0.5)
    quad = np.mean((pts[:, 0] > 0) & (pts[:, 1] > 0))
    sd = math.sqrt(0.25 * 0.75 / len(pts))
    assert abs(inner - 0.25) < 4 * sd and abs(quad - 0.25) < 4 * sd


def test_sunflower_pattern_radii_and_golden_angle():
    """Sunflower: r_a = sqrt((a + 1/2) / M) and consecutive azimuths a golden angle
    pi (3 - sqrt 5) apart; the turn of the whole pattern is shared by every pixel unless
    drawn per pixel."""
    w = refracting_w(rays_per_pixel=8)
    ap = I.workload_pupil(w)
    assert not ap.per_pixel
    pts = O.aperture_points(w, ap, 3, 2)
    M = 8
    np.testing.assert_allclose(np.hypot(pts[:, 0], pts[:, 1]), np.sqrt((np.arange(M) + 0.5) / M), rtol=1e-14)
    ang = np.unwrap(np.arctan2(pts[:, 1], pts[:, 0]))
    dphi = np.mod(np.diff(ang), 2 * np.pi)
    np.testing.assert_allclose(dphi, np.pi * (3 - np.sqrt(5.0)), rtol=1e-12)
    np.testing.assert_array_equal(pts, O.aperture_points(w, ap, 0, 0))
    per = I.Aperture("sunflower", M, seed=0, per_pixel=True)
    a0, a1 = O.aperture_points(w, per, 0, 0), O.aperture_points(w, per, 1, 0)
    assert not np.allclose(a0, a1)
    np.testing.assert_allclose(np.hypot(a1[:, 0], a1[:, 1]), np.hypot(a0[:, 0], a0[:, 1]), rtol=1e-14)


def test_hexagonal_filling_is_a_hex_lattice_in_the_disk():
    """Sec. 2.1 / Sec. 3.2: 13 rays, the points of a hexagonal lattice of spacing 1/2 inside
    the unit disk: radii 0, 1/2 (six) and sqrt(3)/2 (six), every point's nearest neighbour
    exactly 1/2 away, inner ring at multiples of 60 degrees, outer ring 30 degrees off."""
    w = refracting_w(pupil_pattern="hex13", rays_per_pixel=13)
    pts = O.aperture_points(w, I.workload_pupil(w), 4, 1)
    r = np.hypot(pts[:, 0], pts[:, 1])
    np.testing.assert_allclose(np.sort(r), [0.0] + [0.5] * 6 + [math.sqrt(3) / 2] * 6, atol=1e-15)
    dist = np.hypot(pts[:, None, 0] - pts[None, :, 0], pts[:, None, 1] - pts[None, :, 1])
    np.fill_diagonal(dist, np.inf)
    np.testing.assert_allclose(dist.min(axis=1), 0.5, rtol=1e-13)
    deg = np.degrees(np.arctan2(pts[1:, 1], pts[1:, 0])) % 360
    np.testing.assert_allclose(np.sort(deg[r[1:] < 0.6]), [0, 60, 120, 180, 240, 300], atol=1e-12)
    np.testing.assert_allclose(np.sort(deg[r[1:] > 0.6]), [30, 90, 150, 210, 270, 330], atol=1e-12)


def test_named_pattern_drives_the_traced_rays():
    """The traced ray of (u, v, a) leaves the stop point the pattern gives for that pixel."""
    w = small_w(pupil_mm=60.0, f_number=3.0, pupil_pattern="stratified4x4", rays_per_pixel=16)
    ap = I.workload_pupil(w)
    D = w.pupil_mm / w.f_number
    for (u, v, a) in [(0, 0, 0), (10, 3, 7), (20, 6, 15)]:
        xi, eta = O.aperture_points(w, ap, u, v)[a]
        r = O.trace(w, ap, u, v, a)
        np.testing.assert_allclose(r["origin"], [xi * D / 2, -w.pupil_mm, eta * D / 2], atol=1e-14)


def test_ray_generator_telecentric_cone_matches_paper_divergence():
    """Sec. 3.2 / Sec. 4: a 16 mm iris gives a 12.2 degree full divergence.  With the
    working f-number from tan(6.1 deg) = 1/(2N), a telecentric ray from the stop's edge
    makes 6.1 degrees with the chief ray, and every ray of the pixel crosses its image point."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_optics.json")))["telecentric_printer"]
    half = math.radians(gold["full_divergence_large_deg"] / 2)
    N = OP.f_number_for_half_angle(half)
    w = small_w(f_number=N)
    P = np.array([[1.0, 0.0], [0.0, -1.0], [0.0, 0.0]])
    for a in range(3):
        r = O.trace(w, P, 4, 2, a)
        ang = math.degrees(math.acos(r["d0"][1]))
        assert abs(ang - (0.0 if a == 2 else gold["full_divergence_large_deg"] / 2)) < 1e-9
        Q = np.array([pixel_x(w)[4], 0.0, pixel_z(w)[2]])
        t = (Q[1] - r["origin"][1]) / r["d0"][1]
        np.testing.assert_allclose(r["origin"] + t * r["d0"], Q, atol=1e-12)


# --- a2: refraction stage -----------------------------------------------------------------
def _rays(w, P):
    out = []
    for v in range(w.nv):
        for u in range(w.nu):
            for a in range(P.shape[0]):
                out.append(O.trace(w, P, u, v, a))
    return out


def test_snell_invariants_across_coaxial_cylinders():
    """For cylinders about z, n d_z and n (x d_y - y d_x) are conserved by refraction and
    along straight segments; hit points lie on the surfaces and on the incoming lines."""
    # a thick wall (R_in = 3, R_o = 6): rays with n_glass R_in < b < R_o only cross the glass
    w = refracting_w(nu=15, pixel_u_mm=0.9, nv=5, pixel_v_mm=1.3, n_glass=1.52, n_resin=1.43,
                     r_inner_mm=3.0, wall_mm=3.0)
    P = pupil_samples("disk", 5, seed=9)
    Ro, Ri = w.r_inner_mm + w.wall_mm, w.r_inner_mm
    n0, n1, n2 = w.n_outside, w.n_glass, w.n_resin
    seen = {-1: 0, 0: 0, 1: 0, 2: 0}
    for r in _rays(w, P):
        seen[r["status"]] += 1
        if r["status"] == -1:
            # total internal reflection at the glass/resin surface (n_glass > n_resin):
            # the ray is dropped; it must really be beyond the critical angle
            p1, d1 = r["p1"], r["d1"]
            t_near = None
            o2 = p1[:2]
            dd = d1[:2]
            a2, b2, c2 = dd @ dd, 2 * o2 @ dd, o2 @ o2 - Ri * Ri
            t_near = (-b2 - math.sqrt(b2 * b2 - 4 * a2 * c2)) / (2 * a2)
            e = p1 + t_near * d1
            cos_i = abs(e[0] * d1[0] + e[1] * d1[1]) / Ri
            assert n1 * math.sqrt(1 - cos_i ** 2) > n2
            continue
        if r["status"] < 1:
            continue
        o, d0, p1, d1 = r["origin"], r["d0"], r["p1"], r["d1"]
        assert abs(np.linalg.norm(d1) - 1) < 1e-14
        assert abs(math.hypot(p1[0], p1[1]) - Ro) < 1e-12
        t = np.dot(p1 - o, d0)
        np.testing.assert_allclose(o + t * d0, p1, atol=1e-12)
        assert abs(n0 * d0[2] - n1 * d1[2]) < 1e-14
        Lz = lambda p, d: p[0] * d[1] - p[1] * d[0]
        assert abs(n0 * Lz(o, d0) - n1 * Lz(p1, d1)) < 1e-12
        if r["status"] != 2:
            continue
        e, d2, ex = r["e"], r["d2"], r["exit"]
        assert abs(np.linalg.norm(d2) - 1) < 1e-14
        assert abs(math.hypot(e[0], e[1]) - Ri) < 1e-12
        assert abs(math.hypot(ex[0], ex[1]) - Ri) < 1e-12
        t = np.dot(e - p1, d1)
        assert t > 0
        np.testing.assert_allclose(p1 + t * d1, e, atol=1e-12)
        np.testing.assert_allclose(e + r["ell"] * d2, ex, atol=1e-12)
        assert abs(n1 * d1[2] - n2 * d2[2]) < 1e-14
        assert abs(n0 * Lz(o, d0) - n2 * Lz(e, d2)) < 1e-12
        assert e[0] * d2[0] + e[1] * d2[1] < 0          # heads into the resin
        assert r["k"] == math.ceil(r["ell"] / (w.step_vox * w.voxel_mm) - 1e-9)
    assert seen[-1] > 0 and seen[0] > 0 and seen[1] > 0 and seen[2] > 0


def _fresnel_angles(ti, tt):
    """Textbook angle form of the unpolarised Fresnel transmission."""
    if ti == 0.0:
        return None
    rs = (math.sin(ti - tt) / math.sin(ti + tt)) ** 2
    rp = (math.tan(ti - tt) / math.tan(ti + tt)) ** 2
    return 1.0 - 0.5 * (rs + rp)


def test_fresnel_matches_angle_form_and_scalar_snell():
    w = refracting_w(nu=15, pixel_u_mm=0.8, n_glass=1.52, n_resin=1.43)
    P = pupil_samples("disk", 5, seed=9)
    Ro, Ri = w.r_inner_mm + w.wall_mm, w.r_inner_mm
    checked = 0
    for r in _rays(w, P):
        if r["status"] != 2:
            continue
        for (p, R, din, dout, n1, n2, T) in [(r["p1"], Ro, r["d0"], r["d1"], w.n_outside, w.n_glass, r["t1"]),
                                              (r["e"], Ri, r["d1"], r["d2"], w.n_glass, w.n_resin, r["t2"])]:
            nrm = np.array([p[0] / R, p[1] / R, 0.0])
            ti = math.atan2(np.linalg.norm(np.cross(din, nrm)), abs(np.dot(din, nrm)))
            tt = math.atan2(np.linalg.norm(np.cross(dout, nrm)), abs(np.dot(dout, nrm)))
            assert abs(n1 * math.sin(ti) - n2 * math.sin(tt)) < 1e-12
            # refracted ray stays in the plane of incidence
            assert abs(np.dot(np.cross(din, nrm), dout)) < 1e-12
            ref = _fresnel_angles(ti, tt)
            if ref is not None and ti > 1e-3:
                assert abs(T - ref) < 1e-9
                checked += 1
    assert checked > 50


def test_fresnel_normal_incidence():
    """The ray through the axis meets both surfaces head-on: T = 1 - ((n1-n2)/(n1+n2))^2."""
    w = refracting_w(pupil_mm=100.0, f_number=INF, pupil_pattern="chief", rays_per_pixel=1)
    r = O.trace(w, CHIEF, (w.nu - 1) // 2, (w.nv - 1) // 2, 0)
    n0, n1, n2 = w.n_outside, w.n_glass, w.n_resin
    assert r["status"] == 2
    assert abs(r["t1"] - (1 - ((n0 - n1) / (n0 + n1)) ** 2)) < 1e-15
    assert abs(r["t2"] - (1 - ((n1 - n2) / (n1 + n2)) ** 2)) < 1e-15
    np.testing.assert_allclose(r["d2"], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(r["e"], [0, -w.r_inner_mm, 0], atol=1e-14)
    assert abs(r["ell"] - 2 * w.r_inner_mm) < 1e-13


# --- a4/a5: operators ---------------------------------------------------------------------
def test_adjoint_identity_refracting_finite_etendue():
    """<A g, V> = <g, P V>: the dose operator is the exact transpose of the projection."""
    w = refracting_w(nx=17, ny=16, nz=9, nu=11, nv=5, pixel_u_mm=0.9, pixel_v_mm=0.7, n_angles=5,
                     r_inner_mm=3.0, wall_mm=0.8)
    P = pupil_samples("disk", 5, seed=4)
    rng = np.random.default_rng(0)
    V = rng.random(w.vol_shape)
    g = rng.random(w.proj_shape)
    lhs = np.sum(O.forward(w, g, P) * V)
    rhs = np.sum(g * O.adjoint(w, V, P))
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)


def test_dose_matrix_is_transpose_of_projection_matrix():
    w = refracting_w(nx=8, ny=8, nz=4, nu=5, nv=3, pixel_u_mm=0.5, pixel_v_mm=0.5, n_angles=3,
                     r_inner_mm=1.2, wall_mm=0.3, rays_per_pixel=2, pupil_pattern="sunflower", voxel_mm=0.5)
    P = pupil_samples("disk", 2, seed=1)
    nvox, npix = int(np.prod(w.vol_shape)), int(np.prod(w.proj_shape))
    At = np.zeros((npix, nvox))
    for i in range(nvox):
        e = np.zeros(nvox)
        e[i] = 1.0
        At[:, i] = O.adjoint(w, e.reshape(w.vol_shape), P).ravel()
    A = np.zeros((nvox, npix))
    for i in range(npix):
        e = np.zeros(npix)
        e[i] = 1.0
        A[:, i] = O.forward(w, e.reshape(w.proj_shape), P).ravel()
    assert np.count_nonzero(At) > 100
    np.testing.assert_allclose(A, At.T, rtol=0, atol=1e-15)


def _brute_pixel(w, V, P, theta, v, u, sub=256):
    """Independent fine-step integral of trilinear(V) along each traced in-resin segment,
    interpolated with scipy's map_coordinates (order 1, zero outside the grid)."""
    h = w.voxel_mm
    total = 0.0
    for a in range(P.shape[0]):
        r = O.trace(w, P, u, v, a)
        if r["status"] != 2:
            continue
        ell = r["ell"]
        K = int(math.ceil(ell / (h / sub)))
        dl = ell / K
        s = (np.arange(K) + 0.5) * dl
        pts = r["e"][None, :] + s[:, None] * r["d2"][None, :]
        c, sn = math.cos(theta), math.sin(theta)
        xr = c * pts[:, 0] - sn * pts[:, 1]
        yr = sn * pts[:, 0] + c * pts[:, 1]
        coords = [pts[:, 2] / h + (w.nz - 1) / 2, yr / h + (w.ny - 1) / 2, xr / h + (w.nx - 1) / 2]
        vals = map_coordinates(V, coords, order=1, mode="grid-constant", cval=0.0)
        total += r["t1"] * r["t2"] / P.shape[0] * np.sum(np.exp(-w.mu_per_mm * s) * vals) * dl
    return total


def test_brute_force_fine_step_convergence():
    w0 = refracting_w(nx=12, ny=12, nz=10, nu=8, nv=6, pixel_u_mm=0.45, pixel_v_mm=0.45, n_angles=4,
                      r_inner_mm=2.2, wall_mm=0.5, pupil_mm=30.0, f_number=3.0, rays_per_pixel=3,
                      mu_per_mm=0.3)
    P = pupil_samples("disk", 3, seed=2)
    V = np.random.default_rng(5).random(w0.vol_shape)
    th = default_angles(w0.n_angles)
    pix = [(0, 3, 3), (1, 2, 4), (2, 4, 1), (3, 1, 6), (1, 5, 3)]
    ref = np.array([_brute_pixel(w0, V, P, th[k], v, u) for (k, v, u) in pix])
    assert np.all(ref > 0)
    errs = []
    for step in (0.5, 0.125, 1.0 / 64):
        w = w0.scaled(step_vox=step)
        got = O.adjoint_pixels(w, V, P, pix)
        errs.append(np.max(np.abs(got - ref) / ref))
    # midpoint sums converge on the fine integral as the step shrinks
    assert errs[2] < 2e-5
    assert errs[1] < 5e-4
    assert errs[0] < 5e-3
    assert errs[2] < errs[1] < errs[0]


# --- paper numbers ------------------------------------------------------------------------
def test_paper_printed_optics_numbers():
    gold = json.load(open(os.path.join(GOLDEN, "paper_optics.json")))
    nt = gold["non_telecentric_printer"]
    m = OP.magnification(nt["image_pixel_mm"], nt["dmd_pitch_mm"])
    assert abs(m - 5.0) < 1e-12
    assert abs(OP.thin_lens_image_distance(nt["focal_length_mm"], m) - nt["focus_distance_mm"]) < 0.05
    width = nt["dmd_columns"] * nt["image_pixel_mm"]
    assert abs(nt["focus_distance_mm"] / nt["throw_ratio"] - width) / width < 1e-3
    assert abs(nt["downsample"] * nt["image_pixel_mm"] - nt["min_voxel_mm"]) < 1e-12
    tc = gold["telecentric_printer"]
    assert abs(tc["downsample"] * tc["pixel_mm"] - tc["min_voxel_mm"]) < 1e-12
    # both printed divergences come from one stop-to-image distance
    d = tc["iris_large_mm"] / (2 * math.tan(math.radians(tc["full_divergence_large_deg"] / 2)))
    assert abs(OP.full_divergence_deg(tc["iris_small_mm"], d) - tc["full_divergence_small_deg"]) < 0.05
    et = gold["etendue"]
    got = OP.etendue_sr_mm2(et["pixel_mm"], et["full_divergence_deg"])
    assert abs(got - et["etendue_sr_mm2"]) / et["etendue_sr_mm2"] < 1e-3


# --- optimiser and loss (readings) ---------------------------------------------------------
def test_osmo_fixed_point_and_nonnegativity():
    f = np.array([1.0, 0.0, 1.0, 1.0, 0.0])
    ident = lambda x: x.copy()
    g, dn, m, err, ver = OS.osmo(f, ident, ident, n_iter=5)
    assert len(err) == 1 and err[0] == 0.0
    np.testing.assert_array_equal(m, f)
    rng = np.random.default_rng(0)
    M = rng.random((4, 5))
    g, dn, m, err, ver = OS.osmo(f, lambda x: M @ x - 0.8, lambda y: M.T @ y, n_iter=6)
    assert np.all(m >= 0) and np.all(g >= 0) and dn.max() == 1.0
    assert np.all(np.isfinite(err))


# A two-voxel, two-pixel toy printer: dose = B g, projection = B^T m.  Its iterates are
# worked out by hand below (exact fractions), so a dropped term, a wrong sign or a
# transposed operator in either iteration changes them.
B_TOY = np.array([[2.0, 1.0], [1.0, 1.0]])


def test_osmo_two_iterations_by_hand():
    """Object-space iteration on the toy printer, f = (1, 1/2), m0 = f:
    g0 = B^T m0 = (5/2, 3/2); d0 = B g0 = (13/2, 4); dn0 = (1, 8/13); E0 = (3/26)/(3/2) = 1/13;
    m1 = m0 + f - dn0 = (1, 5/13).  g1 = (31/13, 18/13); d1 = (80/13, 49/13); dn1 = (1, 49/80);
    E1 = (9/80)/(3/2) = 3/40; m2 = (1, 5/13 + 1/2 - 49/80) = (1, 283/1040)."""
    f = np.array([1.0, 0.5])
    g, dn, m, err, _ = OS.osmo(f, lambda x: B_TOY.T @ x, lambda y: B_TOY @ y, n_iter=1, tol=0.0)
    np.testing.assert_allclose(g, [2.5, 1.5], rtol=1e-15)
    np.testing.assert_allclose(dn, [1.0, 8.0 / 13.0], rtol=1e-15)
    np.testing.assert_allclose(err, [1.0 / 13.0], rtol=1e-14)
    np.testing.assert_allclose(m, [1.0, 5.0 / 13.0], rtol=1e-15)
    g, dn, m, err, _ = OS.osmo(f, lambda x: B_TOY.T @ x, lambda y: B_TOY @ y, n_iter=2, tol=0.0)
    np.testing.assert_allclose(g, [31.0 / 13.0, 18.0 / 13.0], rtol=1e-15)
    np.testing.assert_allclose(dn, [1.0, 49.0 / 80.0], rtol=1e-15)
    np.testing.assert_allclose(err, [1.0 / 13.0, 3.0 / 40.0], rtol=1e-14)
    np.testing.assert_allclose(m, [1.0, 283.0 / 1040.0], rtol=1e-14)


def test_osmo_model_clamp_by_hand():
    """f = (1, 0): g0 = (2, 1), d0 = (5, 3), dn0 = (1, 3/5), E0 = 3/5; the update would take
    the void voxel's model to -3/5 and the clamp holds it at 0, so m1 = f."""
    f = np.array([1.0, 0.0])
    g, dn, m, err, _ = OS.osmo(f, lambda x: B_TOY.T @ x, lambda y: B_TOY @ y, n_iter=1, tol=0.0)
    np.testing.assert_allclose(dn, [1.0, 0.6], rtol=1e-15)
    np.testing.assert_allclose(err, [0.6], rtol=1e-15)
    np.testing.assert_array_equal(m, [1.0, 0.0])


def test_osmo_normalises_by_the_resin_maximum():
    """The dose is normalised by its maximum over the resin voxels only: with voxel 0
    outside the resin, dn0 = d0 / d0[1] = (13/8, 1) for the toy's f = (1, 1/2)."""
    f = np.array([1.0, 0.5])
    _, dn, _, _, _ = OS.osmo(f, lambda x: B_TOY.T @ x, lambda y: B_TOY @ y, n_iter=1, tol=0.0,
                             resin=np.array([False, True]))
    np.testing.assert_allclose(dn, [13.0 / 8.0, 1.0], rtol=1e-15)


def test_osmo_projections_closed_form():
    """Projection-space iteration on the toy printer B = [[2, 1], [0, 1]] (the second voxel
    is reached by the second pixel only), f = (1, 0), g0 = (1, 1), alpha = 1:
    g_k = (1, c_k) with c_{k+1} = c_k - c_k / (2 + c_k) and E_k = c_k / (2 + c_k):
    c = 1, 2/3, 5/12; E = 1/3, 1/4.  The fixed point g = (1, 0) prints f exactly (E = 0).
    With alpha = 1/2 the displacement of the first step halves: c1 = 1 - 1/6."""
    f = np.array([1.0, 0.0])
    B = np.array([[2.0, 1.0], [0.0, 1.0]])
    project, dose = (lambda x: B.T @ x), (lambda y: B @ y)
    g, dn, err = OS.osmo_projections(f, np.array([1.0, 1.0]), project, dose, n_iter=2, alpha=1.0)
    np.testing.assert_allclose(err, [1.0 / 3.0, 1.0 / 4.0], rtol=1e-15)
    np.testing.assert_allclose(g, [1.0, 5.0 / 12.0], rtol=1e-15)
    g, _, _ = OS.osmo_projections(f, np.array([1.0, 1.0]), project, dose, n_iter=1, alpha=0.5)
    np.testing.assert_allclose(g, [1.0, 5.0 / 6.0], rtol=1e-15)
    g, dn, err = OS.osmo_projections(f, np.array([1.0, 0.0]), project, dose, n_iter=3)
    np.testing.assert_array_equal(g, [1.0, 0.0])
    np.testing.assert_array_equal(err, [0.0, 0.0, 0.0])


def test_threshold_adam_by_hand():
    """Thresholded-loss Adam continuation on the toy printer B = [[2, 1], [1, 1]] (dose B g,
    projection B^T x), f = (1, 0), g0 = (1, 1), d_l = 1/2, d_h = 1, step 0.8:
    A g0 = (3, 2), the part's mean dose 3, so g = (1/3, 1/3) and lr = 0.8 / 3 = 4/15.
    Iteration 1: D = (1, 2/3); only the void voxel is over d_l: L = (1/6)^2 = 1/36,
    dL/dD = (0, 1/3), grad = B^T (0, 1/3) = (1/3, 1/3).  Adam's first bias-corrected step is
    lr sign(grad) (m^ = grad, v^ = grad^2), so g1 = (1/3 - 4/15, ...) = (1/15, 1/15).
    Iteration 2: D = (1/5, 2/15); now the part is under-dosed: L = (4/5)^2 = 16/25,
    grad = B^T (-8/5, 0) = (-16/5, -8/5); m = (-0.29, -0.13), v = (0.010351, 0.002671),
    bias corrections 0.19 and 0.001999: g2 = 1/15 + (4/15)(0.670748..., 0.591916...)
    = (0.2455329..., 0.2245106...)."""
    B = np.array([[2.0, 1.0], [1.0, 1.0]])
    project, dose = (lambda x: B.T @ x), (lambda y: B @ y)
    f = np.array([1.0, 0.0])
    g, D, L = OS.threshold_adam(f, np.array([1.0, 1.0]), project, dose, n_iter=1, step=0.8, d_l=0.5, d_h=1.0)
    np.testing.assert_allclose(L, [1.0 / 36.0], rtol=1e-14)
    np.testing.assert_allclose(D, [1.0, 2.0 / 3.0], rtol=1e-15)
    np.testing.assert_allclose(g, [1.0 / 15.0, 1.0 / 15.0], rtol=1e-10)
    g, D, L = OS.threshold_adam(f, np.array([1.0, 1.0]), project, dose, n_iter=2, step=0.8, d_l=0.5, d_h=1.0)
    np.testing.assert_allclose(L, [1.0 / 36.0, 16.0 / 25.0], rtol=1e-9)
    np.testing.assert_allclose(D, [0.2, 2.0 / 15.0], rtol=1e-9)
    np.testing.assert_allclose(g, [0.24553290433, 0.22451061528], rtol=1e-9)
    # the projection bound: a step that would go below zero stops at zero
    g, _, _ = OS.threshold_adam(f, np.array([1.0, 1.0]), project, dose, n_iter=1, step=3.0, d_l=0.5, d_h=1.0)
    np.testing.assert_array_equal(g, [0.0, 0.0])


def test_osmo_stops_on_the_voxel_error_rate():
    """The stop reads Sec. 2.7's 'absolute relative error below 0.5 %' as the voxel error
    rate V of the normalised dose: the loop ends after the first iteration whose V is below
    tol, and the dose error E is reported beside it.  On the toy printer with f = (1, 0),
    V0 = 0 (the threshold between 3/5 and 1 separates the voxels) while E0 = 3/5, so a
    0.5 % stop on V ends after one iteration and a 0.5 % stop on E does not."""
    f = np.array([1.0, 0.0])
    project, dose = (lambda x: B_TOY.T @ x), (lambda y: B_TOY @ y)
    _, _, _, err, ver = OS.osmo(f, project, dose, n_iter=4, tol=0.005)
    assert len(err) == 1 and ver[0] == 0.0 and abs(err[0] - 0.6) < 1e-15
    _, _, _, err, ver = OS.osmo(f, project, dose, n_iter=4, tol=0.005, stop="error")
    assert len(err) == 4 and np.all(err > 0.005)


def test_osmo_relaxed_step_scales_the_model_update():
    """The over-relaxed update m <- max(0, m + beta (f - dn)): away from the clamp one
    iteration moves the model beta times as far as the plain one, along the same
    direction; the fixed point f (dn = f) is kept for any beta."""
    f = np.array([1.0, 1.0, 0.8, 1.0])
    tilt = np.array([1.0, 1.05, 0.9, 1.1])
    project = lambda x: tilt * x
    dose = lambda y: y.copy()
    _, _, m1, _, _ = OS.osmo(f, project, dose, n_iter=1, tol=0.0)
    _, _, m3, _, _ = OS.osmo(f, project, dose, n_iter=1, tol=0.0, beta=3.0)
    assert np.all(m1 > 0) and np.all(m3 > 0)
    np.testing.assert_allclose(m3 - f, 3.0 * (m1 - f), rtol=0, atol=1e-15)
    assert np.abs(m1 - f).max() > 0.05
    ident = lambda x: x.copy()
    fb = np.array([1.0, 0.0, 1.0])
    _, _, m, err, _ = OS.osmo(fb, ident, ident, n_iter=3, tol=0.0, beta=4.0)
    np.testing.assert_array_equal(m, fb)
    assert np.all(np.array(err) == 0.0)


def test_osmo_momentum_adds_the_previous_step():
    """Heavy-ball momentum: from rest the first iteration is the plain one; from a model
    m1 with predecessor m0, away from the clamp, the iterate differs from the
    momentum-free one from m1 by exactly mu (m1 - m0)."""
    f = np.array([1.0, 1.0, 0.8, 1.0])
    tilt = np.array([1.0, 1.05, 0.9, 1.1])
    project = lambda x: tilt * x
    dose = lambda y: y.copy()
    _, _, m1, _, _ = OS.osmo(f, project, dose, n_iter=1, tol=0.0, beta=2.0)
    _, _, m1_mu, _, _ = OS.osmo(f, project, dose, n_iter=1, tol=0.0, beta=2.0, mu=0.5)
    np.testing.assert_array_equal(m1_mu, m1)
    _, _, m2, _, _ = OS.osmo(f, project, dose, n_iter=1, tol=0.0, beta=2.0, m0=m1)
    _, _, m2_mu, _, _ = OS.osmo(f, project, dose, n_iter=1, tol=0.0, beta=2.0, mu=0.5, m0=m1, m_prev=f)
    assert np.all(m2 > 0) and np.all(m2_mu > 0)
    np.testing.assert_allclose(m2_mu - m2, 0.5 * (m1 - f), rtol=0, atol=1e-15)
    assert np.abs(m1 - f).max() > 0.05
    _, _, m2_two, _, _ = OS.osmo(f, project, dose, n_iter=2, tol=0.0, beta=2.0, mu=0.5)
    np.testing.assert_allclose(m2_two, m2_mu, rtol=0, atol=1e-15)


# --- lens train (Sec. 2.1, 2.6.2) -------------------------------------------------------
def _lens_w(surfaces, **kw):
    L = I.LensTrain(surfaces=tuple(surfaces), object_y_mm=-100.0, magnification=-1.0, aim_mm=50.0)
    return I.TINY.scaled(lens=L, **kw)


def test_thick_lens_focus_matches_the_lensmaker_formula():
    """A paraxial ray parallel to the axis through a biconvex thick lens crosses the axis at
    the back focal distance f (1 - (n - 1) t / (n R1)), 1/f = (n - 1)(1/R1 - 1/R2 +
    (n - 1) t / (n R1 R2))."""
    R1, R2, t, n = 50.0, -50.0, 5.0, 1.5
    w = _lens_w([I.Surface(0.0, R1, n, 20.0), I.Surface(t, R2, 1.0, 20.0)])
    f = 1.0 / ((n - 1) * (1 / R1 - 1 / R2 + (n - 1) * t / (n * R1 * R2)))
    bfd = f * (1 - (n - 1) * t / (n * R1))
    ok, o, d = O.lens_trace(w, [0.01, -50.0, 0.0], [0.0, 1.0, 0.0])
    assert ok
    y_cross = o[1] - o[0] * d[1] / d[0]
    assert abs((y_cross - t) - bfd) < 1e-5 * f


def test_plane_parallel_plate_shifts_without_deviating():
    """A tilted ray through a plate of thickness t and index n leaves parallel to itself,
    displaced by t sin(a) (1 - cos(a) / sqrt(n^2 - sin^2(a)))."""
    t, n, a = 3.0, 1.6, 0.3
    w = _lens_w([I.Surface(0.0, I.INF, n, 50.0), I.Surface(t, I.INF, 1.0, 50.0)])
    d0 = np.array([np.sin(a), np.cos(a), 0.0])
    o0 = np.array([0.0, -10.0, 0.0])
    ok, o, d = O.lens_trace(w, o0, d0)
    assert ok and np.allclose(d, d0, atol=1e-15)
    # distance between the exit line and the undeviated line
    shift = np.linalg.norm(np.cross(o - o0, d0))
    assert abs(shift - t * np.sin(a) * (1 - np.cos(a) / np.sqrt(n * n - np.sin(a) ** 2))) < 1e-12


def test_lens_train_conserves_the_skew_invariant_and_blocks_outside_apertures():
    """Refraction at surfaces symmetric about the optical axis conserves n (z d_x - x d_z);
    a ray outside a clear aperture is blocked."""
    L = I.telecentric_relay()
    w = I.TINY.scaled(lens=L)
    rng = np.random.default_rng(3)
    for _ in range(20):
        o0 = np.array([rng.uniform(-3, 3), L.object_y_mm, rng.uniform(-3, 3)])
        d0 = np.array([rng.uniform(-0.05, 0.05), 1.0, rng.uniform(-0.05, 0.05)])
        d0 /= np.linalg.norm(d0)
        ok, o, d = O.lens_trace(w, o0, d0)
        if not ok:
            continue
        L0 = o0[2] * d0[0] - o0[0] * d0[2]
        L1 = o[2] * d[0] - o[0] * d[2]
        assert abs(L1 - L0) < 1e-12 and abs(np.linalg.norm(d) - 1) < 1e-14
    ok, _, _ = O.lens_trace(w, [0.0, L.object_y_mm, 0.0], [0.2, 1.0, 0.0] / np.linalg.norm([0.2, 1.0, 0.0]))
    assert not ok                                    # 0.2 rad misses the 12.7 mm lens / 8 mm iris


def test_telecentric_relay_images_and_stays_telecentric():
    """Sec. 2.6.2's printer as a 4f relay: near the axis every aperture ray of a pixel
    lands on the pixel's image point in y = 0 and the chief ray leaves parallel to the
    axis (unit magnification, image-space telecentric)."""
    w = I.TINY.scaled(lens=I.telecentric_relay(iris_diameter_mm=2.5), pupil_pattern="hex13", rays_per_pixel=13,
                      f_number=4.0)
    pup = I.workload_pupil(w)
    for u, v in ((32, 32), (33, 31)):
        q = np.array([(u - (w.nu - 1) / 2) * w.pixel_u_mm, 0.0, (v - (w.nv - 1) / 2) * w.pixel_v_mm])
        for a in range(13):
            r = O.trace(w, pup, u, v, a)
            o, d = r["origin"], r["d0"]
            p = o - o[1] / d[1] * d
            assert np.linalg.norm(p - q) < 2e-3, (u, v, a)
            if a == 0:
                assert abs(d[0]) < 1e-4 and abs(d[2]) < 1e-4


# --- Radon-method baseline (Sec. 2.3) ---------------------------------------------------
def test_ramlak_frequency_response_is_the_ramp():
    """The band-limited ramp kernel's discrete-time Fourier transform is |omega| / (2 pi) on
    [-pi, pi] (Kak & Slaney); truncated to 4096 taps it stays within 3e-5 of it."""
    from oracle import radon as RD
    h = RD.ramlak_taps(4096)
    k = np.arange(1, 4096)
    for om in (0.0, 0.3, np.pi / 4, np.pi / 2, 2.0, np.pi):
        H = h[0] + 2.0 * np.sum(h[1:] * np.cos(om * k))
        assert abs(H - om / (2 * np.pi)) < 3e-5, om


def test_ramlak_filtered_backprojection_reconstructs_a_disk():
    """Textbook filtered backprojection: the analytic parallel-beam sinogram of a unit disk
    (chords 2 sqrt(R^2 - s^2)), filtered by the oracle and backprojected over 180 angles,
    gives 1 inside the disk and ~0 outside."""
    from oracle import radon as RD
    n, tau, R = 129, 0.5, 20.0
    s = (np.arange(n) - (n - 1) / 2) * tau
    sino = np.where(np.abs(s) < R, 2 * np.sqrt(np.maximum(R * R - s * s, 0.0)), 0.0)
    na = 180
    th = np.pi * np.arange(na) / na
    q = RD.ramlak_filter(np.tile(sino, (na, 1)), tau)
    X, Y = np.meshgrid(s, s)
    rec = np.zeros_like(X)
    for a in range(na):
        rec += np.interp(X * np.cos(th[a]) + Y * np.sin(th[a]), s, q[a], left=0.0, right=0.0)
    rec *= np.pi / na
    r = np.hypot(X, Y)
    assert np.abs(rec[r < 0.8 * R] - 1.0).max() < 0.01
    ring = (r > 1.2 * R) & (r < 1.5 * R)
    assert np.abs(rec[ring]).mean() < 0.02
    clipped = RD.ramlak_filter(np.tile(sino, (2, 1)), tau, clamp=True)
    assert clipped.min() == 0.0 and np.array_equal(clipped[0], np.maximum(q[0], 0.0))


def test_threshold_loss_gradient_central_differences():
    rng = np.random.default_rng(1)
    D = rng.random(200) * 1.4
    f = (rng.random(200) < 0.4).astype(np.float64)
    L, g = OS.threshold_loss(D, f, 0.9, 1.0)
    eps = 1e-6
    for i in range(0, 200, 7):
        Dp, Dm = D.copy(), D.copy()
        Dp[i] += eps
        Dm[i] -= eps
        fd = (OS.threshold_loss(Dp, f, 0.9, 1.0)[0] - OS.threshold_loss(Dm, f, 0.9, 1.0)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7
    L0, g0 = OS.threshold_loss(np.where(f > 0, 1.2, 0.5), f, 0.9, 1.0)
    assert L0 == 0.0 and np.all(g0 == 0.0)


def test_voxel_error_rate_small_cases():
    """VER by hand: doses whose best threshold is known."""
    f = np.array([1, 1, 0, 0, 1, 0], dtype=np.float32)
    resin = np.ones(6, dtype=bool)
    d = np.array([0.9, 1.0, 0.2, 0.1, 0.95, 0.3], dtype=np.float32)
    ver, i = OS.voxel_error_rate(d, f, resin)
    assert ver == 0.0 and 0.3 < i / 1024 <= 0.9
    d2 = np.array([0.9, 0.2, 0.5, 0.1, 1.0, 0.3], dtype=np.float32)   # one in-part voxel too dim
    ver2, _ = OS.voxel_error_rate(d2, f, resin)
    assert abs(ver2 - 1 / 6) < 1e-12
    resin2 = np.array([1, 0, 1, 1, 1, 1], dtype=bool)                  # ...unless it is outside the resin
    ver3, _ = OS.voxel_error_rate(d2, f, resin2)
    assert ver3 == 0.0


def test_conv3d_oracle_against_scalar_loops():
    """The oracle convolution against the definition written out as scalar loops."""
    from oracle import conv3d as C
    rng = np.random.default_rng(4)
    D, H, W, Cin, Cout = 3, 4, 5, 2, 3
    x = rng.standard_normal((D, H, W, Cin))
    w = rng.standard_normal((Cout, 27, Cin))
    b = rng.standard_normal(Cout)
    y = C.conv3d(x, w, b, relu=False)
    for (z, yy, xx) in [(0, 0, 0), (1, 2, 3), (2, 3, 4), (0, 3, 2)]:
        for co in range(Cout):
            acc = b[co]
            t = 0
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        zi, yi, xi = z + dz, yy + dy, xx + dx
                        if 0 <= zi < D and 0 <= yi < H and 0 <= xi < W:
                            acc += sum(x[zi, yi, xi, ci] * w[co, t, ci] for ci in range(Cin))
                        t += 1
            assert abs(y[z, yy, xx, co] - acc) < 1e-12
    # 1x1x1 is a per-voxel matrix product
    w1 = rng.standard_normal((Cout, 1, Cin))
    np.testing.assert_allclose(C.conv3d(x, w1), x @ w1[:, 0, :].T, rtol=1e-14)


def test_unattenuated_projection_removes_fresnel_and_absorption():
    """Sec. 2.4's projection as printed: with one ray per pixel it equals the attenuated
    projection at mu = 0 divided by the ray's Fresnel product T1 T2."""
    w = refracting_w(pupil_pattern="chief", rays_per_pixel=1, f_number=INF, mu_per_mm=0.4, n_angles=3)
    V = np.random.default_rng(6).random(w.vol_shape)
    y_lit = O.adjoint(w, V, CHIEF, unattenuated=True)
    y_mu0 = O.adjoint(w.scaled(mu_per_mm=0.0), V, CHIEF)
    for (v, u) in [(3, 10), (1, 4), (5, 16), (0, 0)]:
        r = O.trace(w, CHIEF, u, v, 0)
        expect = y_mu0[:, v, u] / (r["t1"] * r["t2"]) if r["status"] == 2 else 0.0 * y_mu0[:, v, u]
        np.testing.assert_allclose(y_lit[:, v, u], expect, rtol=1e-12, atol=1e-14)


def test_export_u8_codes():
    """Clip at mean + 3 sigma, 255 levels, round half to even."""
    g = np.array([0.0, 1.0, 2.0, 3.0, 100.0] + [1.0] * 20)
    codes, c = OS.export_u8(g)
    assert abs(c - (g.mean() + 3 * g.std())) < 1e-12
    assert codes[4] == 255 and codes[0] == 0
    np.testing.assert_array_equal(codes[1:4], np.rint(255 * g[1:4] / c).astype(np.uint8))
    codes2, _ = OS.export_u8(np.array([0.5, 1.5, 1.0, 1.0]))   # c = 1 + 3 * sqrt(1/8)
    assert codes2.dtype == np.uint8 and codes2.max() <= 255


# --- warm-start network reference (oracle/unet_ref.py) -------------------------------------
def _ref_arch():
    return [("enc0a", 16, 16, 27), ("enc0b", 16, 16, 27), ("enc1a", 16, 32, 27), ("enc1b", 32, 32, 27),
            ("enc2a", 32, 64, 27), ("enc2b", 64, 64, 27), ("bota", 64, 128, 27), ("botb", 128, 128, 27),
            ("dec2a", 192, 64, 27), ("dec2b", 64, 64, 27), ("dec1a", 96, 32, 27), ("dec1b", 32, 32, 27),
            ("dec0a", 48, 16, 27), ("dec0b", 16, 16, 27), ("head", 16, 16, 1)]


def test_unet_reference_head_and_loss_in_closed_form():
    """With every convolution weight zero the network is constant: the last decoder layer
    outputs relu(b_dec0b), the head z = W_head relu(b_dec0b) + b_head (channel 0 used), and
    out = in_scale base + z.  Loss, dL/db_head[0] and dL/dW_head[0, c] then have closed forms
    (mean squared error over the first n_angles slices): a wrong head channel, a missing
    input scale, a dropped 1/2 or mean, or a gradient through the wrong channel fails."""
    from oracle import unet_ref
    rng = np.random.default_rng(5)
    arch = _ref_arch()
    weights = {n: (np.zeros((co, t, ci)), np.zeros(co)) for (n, ci, co, t) in arch}
    b_dec = rng.uniform(-1.0, 1.0, 16)
    weights["dec0b"] = (np.zeros((16, 27, 16)), b_dec)
    Wh = rng.standard_normal((16, 1, 16))
    bh = rng.standard_normal(16)
    weights["head"] = (Wh, bh)
    Dp, V, U, A = 8, 8, 8, 6
    x = rng.random((Dp, V, U, 16))
    base = rng.random((A, V, U))
    target = rng.random((A, V, U))
    s = 0.7
    loss, z, grads = unet_ref.loss_and_grads(arch, weights, x, target, A, base, s)
    h = np.maximum(b_dec, 0.0)
    z0 = Wh[0, 0] @ h + bh[0]
    out = s * base + z0
    r = out - target
    assert abs(loss - 0.5 * np.mean(r ** 2)) <= 1e-12 * abs(loss)
    np.testing.assert_allclose(z[..., 0], z0, rtol=1e-12)
    gW, gb = grads["head"]
    np.testing.assert_allclose(gb[0], np.mean(r), rtol=1e-10)
    np.testing.assert_allclose(gb[1:], 0.0, atol=1e-15)
    np.testing.assert_allclose(gW[0, 0], np.mean(r) * h, rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(gW[1:], 0.0, atol=1e-15)
