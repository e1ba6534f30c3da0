"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's callers.

This module holds workload descriptions (printer, vial and grid parameters), binary
target volumes, aperture-stop sample patterns and random fields.  It contains none of
the ray-tracing or dose arithmetic: it only produces the numbers that both the CUDA
path and the CPU oracle are fed with.

The paper's own parts (a 3DBenchy, a 9-fin part, a lettered part) are not available;
seeded constructive-solid-geometry targets of the same kind (solid bodies with thin
features, placed inside the region the refracted rays reach from every angle) stand in
for them.  Every generator is a pure function of its arguments and seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

INF = float("inf")


@dataclass(frozen=True)
class Surface:
    """One rotationally symmetric surface of a lens train on the optical axis (the y axis
    through x = z = 0): vertex at y_mm, radius of curvature radius_mm (centre at
    y_mm + radius_mm; INF = plane), index n_after behind it, clear semi-aperture clear_mm;
    stop: the aperture stop (an iris: a plane that blocks, no refraction)."""

    y_mm: float
    radius_mm: float
    n_after: float
    clear_mm: float
    stop: bool = False


@dataclass(frozen=True)
class LensTrain:
    """Surfaces between the pixel array (at object_y_mm) and the vial, in increasing y.
    Pixel (u, v) sits at Q_uv / magnification in the object plane (Q_uv its nominal image
    point in the best-focus plane y = 0); aperture sample (xi, eta) leaves it with
    direction proportional to (xi r_s / aim_mm, 1, eta r_s / aim_mm), r_s = the stop radius
    (object-space telecentric launch aimed paraxially at the stop)."""

    surfaces: tuple
    object_y_mm: float
    magnification: float
    aim_mm: float


def _abcd(surfaces, n0, y0, y1):
    """Paraxial (height, n * angle) transfer matrix from plane y0 to plane y1 through the
    surfaces between them."""
    M = np.eye(2)
    y, n = y0, n0
    for sf in surfaces:
        M = np.array([[1.0, (sf.y_mm - y) / n], [0.0, 1.0]]) @ M
        if not sf.stop and math.isfinite(sf.radius_mm):
            M = np.array([[1.0, 0.0], [-(sf.n_after - n) / sf.radius_mm, 1.0]]) @ M
        y, n = sf.y_mm, sf.n_after
    return np.array([[1.0, (y1 - y) / n], [0.0, 1.0]]) @ M


def telecentric_relay(lens_radius_mm: float = 38.6, lens_thickness_mm: float = 4.1, n_lens: float = 1.5302,
                      lens_clear_mm: float = 12.7, iris_diameter_mm: float = 16.0, n_air: float = 1.0) -> LensTrain:
    """The telecentric printer of Sec. 2.6.2 as a parameterised 4f relay: two identical
    plano-convex lenses, convex faces towards the iris midway between them, the pixel array
    at the front focal plane of the first and the best-focus plane y = 0 at the back focal
    plane of the second (paraxial), so unit magnification, object and image space
    telecentric.  The paper names the lens (a 75 mm plano-convex singlet) but not its
    prescription; the defaults are a stock 75 mm N-BK7 plano-convex lens (index at 405 nm),
    with which the pixel array lands near the paper's y = -294 mm."""
    R, tc, n = lens_radius_mm, lens_thickness_mm, n_lens
    # first lens: plane face at y = 0 (reference), convex face at y = tc bulging towards +y
    l1 = [Surface(0.0, INF, n, lens_clear_mm), Surface(tc, -R, n_air, lens_clear_mm)]
    # paraxial matrix of the first lens from its plane face to its convex vertex
    M = _abcd(l1, n_air, 0.0, tc)
    f_eff = -n_air / M[1, 0]
    bfd = -M[0, 0] / M[1, 0] * n_air             # convex vertex -> back focus (parallel input)
    ffd = -M[1, 1] / M[1, 0] * n_air             # front focus -> plane face (parallel output)
    stop_y = tc + bfd
    # second lens mirrored about the stop
    l2 = [Surface(2 * stop_y - tc, R, n, lens_clear_mm), Surface(2 * stop_y, INF, n_air, lens_clear_mm)]
    image_y = 2 * stop_y + ffd
    obj_y = -ffd
    shift = -image_y                             # put the image plane at y = 0
    surfs = tuple(Surface(sf.y_mm + shift, sf.radius_mm, sf.n_after, sf.clear_mm, sf.stop)
                  for sf in l1 + [Surface(stop_y, INF, n_air, iris_diameter_mm / 2, True)] + l2)
    return LensTrain(surfaces=surfs, object_y_mm=obj_y + shift, magnification=-1.0, aim_mm=f_eff)


@dataclass(frozen=True)
class Workload:
    """One printer + vial + grid configuration (units: mm, radians, 1/mm).

    Grid: nx*ny*nz voxels of pitch ``voxel_mm``, centred on the vial axis (z).
    Pixel array: nu*nv pixels of pitch pixel_u_mm x pixel_v_mm in the best-focus plane
    y = 0, which contains the rotation axis (Sec. 2.8).  The aperture stop sits
    ``pupil_mm`` in front of the axis on the -y side (INF = telecentric, Sec. 2.6);
    its diameter is pupil_mm / f_number (telecentric: cone half-angle atan(1/(2N))).
    """

    name: str
    nx: int
    ny: int
    nz: int
    voxel_mm: float
    nu: int
    nv: int
    pixel_u_mm: float
    pixel_v_mm: float
    n_angles: int
    pupil_mm: float
    f_number: float
    pupil_pattern: str  # chief | stratified<n>x<n> | sunflower | hex13
    rays_per_pixel: int
    r_inner_mm: float
    wall_mm: float
    n_outside: float
    n_glass: float
    n_resin: float
    mu_per_mm: float
    step_vox: float = 0.5
    target: str = "sphere_cube"
    seed: int = 0
    osmo_iters: int = 10
    lens: Optional[LensTrain] = None   # a lens train replacing the ideal pupil model
    jitter_per_pixel: Optional[bool] = None   # None: per pixel for stratified, shared otherwise

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def proj_shape(self):
        return (self.n_angles, self.nv, self.nu)


# The five workloads of the benchmark spec, named by what they are.  Values the task leaves open
# (c3 vial, c4 pitch/vial, pixel pitch = voxel pitch) follow the readings listed in the
# design notes.
WORKLOADS = {
    "tiny_64cube_90ang_chief": Workload(
        name="tiny_64cube_90ang_chief", nx=64, ny=64, nz=64, voxel_mm=0.2,
        nu=64, nv=64, pixel_u_mm=0.2, pixel_v_mm=0.2, n_angles=90,
        pupil_mm=150.0, f_number=INF, pupil_pattern="chief", rays_per_pixel=1,
        r_inner_mm=6.0, wall_mm=1.0, n_outside=1.0, n_glass=1.47, n_resin=1.50,
        mu_per_mm=0.05, target="sphere_cube", seed=0, osmo_iters=10),
    "mid_256cube_360ang_16rays": Workload(
        name="mid_256cube_360ang_16rays", nx=256, ny=256, nz=256, voxel_mm=0.1,
        nu=256, nv=256, pixel_u_mm=0.1, pixel_v_mm=0.1, n_angles=360,
        pupil_mm=120.0, f_number=4.0, pupil_pattern="stratified4x4", rays_per_pixel=16,
        r_inner_mm=12.5, wall_mm=1.2, n_outside=1.0, n_glass=1.47, n_resin=1.50,
        mu_per_mm=0.03, target="spheres_tori12", seed=0, osmo_iters=30),
    "tall_384x384x512_720ang_8rays": Workload(
        name="tall_384x384x512_720ang_8rays", nx=384, ny=384, nz=512, voxel_mm=0.08,
        nu=384, nv=512, pixel_u_mm=0.08, pixel_v_mm=0.08, n_angles=720,
        pupil_mm=80.0, f_number=4.0, pupil_pattern="sunflower", rays_per_pixel=8,
        r_inner_mm=15.0, wall_mm=1.2, n_outside=1.0, n_glass=1.47, n_resin=1.50,
        mu_per_mm=0.03, target="strut_lattice", seed=0, osmo_iters=30),
    "warmstart_128cube_180ang_4rays": Workload(
        name="warmstart_128cube_180ang_4rays", nx=128, ny=128, nz=128, voxel_mm=0.1,
        nu=128, nv=128, pixel_u_mm=0.1, pixel_v_mm=0.1, n_angles=180,
        pupil_mm=100.0, f_number=4.0, pupil_pattern="sunflower", rays_per_pixel=4,
        r_inner_mm=6.0, wall_mm=1.0, n_outside=1.0, n_glass=1.47, n_resin=1.50,
        mu_per_mm=0.05, target="csg", seed=0, osmo_iters=40),
    "large_768x768x1024_1000ang_4rays": Workload(
        name="large_768x768x1024_1000ang_4rays", nx=768, ny=768, nz=1024, voxel_mm=0.05,
        nu=1024, nv=1024, pixel_u_mm=0.05, pixel_v_mm=0.05, n_angles=1000,
        pupil_mm=100.0, f_number=2.8, pupil_pattern="sunflower", rays_per_pixel=4,
        r_inner_mm=19.0, wall_mm=1.5, n_outside=1.0, n_glass=1.47, n_resin=1.50,
        mu_per_mm=0.02, target="csg_shells", seed=0, osmo_iters=30),
}

TINY = WORKLOADS["tiny_64cube_90ang_chief"]
MID = WORKLOADS["mid_256cube_360ang_16rays"]


# ----------------------------------------------------------------------------------
# aperture-stop sampling: which pattern a projector uses (the points themselves are
# generated inside the CUDA library and, independently, inside the oracle)
# ----------------------------------------------------------------------------------
@dataclass(frozen=True)
class Aperture:
    """The aperture-stop samples of a projector, by name (Sec. 2.1: rays leave points of
    the stop).  pattern: "chief" (one ray, the stop's centre), "stratified" (n x n
    jittered strata, n_rays = n^2), "sunflower" (golden-angle spiral) or "hex13" (the
    paper's hexagonal filling, 13 rays).  seed and per_pixel select the jitter draws.
    Holds no sample positions: both the library and the oracle generate them."""

    pattern: str
    n_rays: int
    seed: int = 0
    per_pixel: bool = False


def workload_pupil(w: Workload) -> Aperture:
    """The workload's aperture pattern.  Stratified jitter is drawn per pixel (the 4 x 4
    'stratified jitter' of the 256^3 workload); the sunflower's turn is shared by every
    pixel, so that ray a of neighbouring pixels leaves nearly the same stop point (set
    jitter_per_pixel to draw it per pixel)."""
    pat = w.pupil_pattern
    kind = "stratified" if pat.startswith("stratified") else pat
    if kind not in ("chief", "stratified", "sunflower", "hex13"):
        raise ValueError(f"unknown pupil pattern {pat!r}")
    if kind == "stratified":
        n = int(pat[len("stratified"):].split("x")[0])
        if n * n != w.rays_per_pixel:
            raise ValueError(f"{pat} needs {n * n} rays, got {w.rays_per_pixel}")
    if kind == "chief" and w.rays_per_pixel != 1:
        raise ValueError("chief pattern has exactly one ray")
    if kind == "hex13" and w.rays_per_pixel != 13:
        raise ValueError("hex13 has 13 rays")
    per_pixel = (kind == "stratified") if w.jitter_per_pixel is None else bool(w.jitter_per_pixel)
    return Aperture(kind, w.rays_per_pixel, w.seed, per_pixel)


def pupil_samples(pattern: str, m: int, seed: int = 0) -> np.ndarray:
    """An explicit (m, 2) float64 list of stop points (xi, eta), passed to a projector in
    place of a named pattern: "chief" = the single point (0, 0); "disk" = m seeded points
    drawn uniformly in the unit disk (rejection from the square)."""
    if pattern == "chief":
        if m != 1:
            raise ValueError("chief pattern has exactly one ray")
        return np.zeros((1, 2))
    if pattern == "disk":
        rng = np.random.default_rng(seed)
        pts = []
        while len(pts) < m:
            x, y = rng.uniform(-1.0, 1.0, size=2)
            if x * x + y * y <= 1.0:
                pts.append((x, y))
        return np.array(pts)
    raise ValueError(f"unknown explicit pupil list {pattern!r}")


# Fin part (Sec. 3: 1 mm fins at a 2.25 mm period, normal to the vial axis, on a base at
# the projector's optical axis), built on a 2 mm base with a 1 mm spine; half-width 4 mm.
FIN_BASE_MM, FIN_GAP0_MM, FIN_PERIOD_MM, FIN_THICK_MM, FIN_HALF_MM = 2.0, 1.25, 2.25, 1.0, 4.0


def fin_bottoms_mm(n_fins: int) -> np.ndarray:
    """z of the lower face of each fin (the base spans z in [0, 2] mm)."""
    return FIN_BASE_MM + FIN_GAP0_MM + FIN_PERIOD_MM * np.arange(n_fins)


def fins_workload(n_fins: int = 9) -> Workload:
    """The non-telecentric printer of Sec. 2.6.1 for the fin part: pupil (ideal lens at the
    aperture stop) 99.5 mm from the axis, chief rays only (low etendue), vial OD 25 / ID
    23.6 mm, 0.216 mm voxels (the paper's minimum after its 4 x 4 downsampling) and pixels
    of the same pitch, 360 angles.  The grid is centred on z = 0 (the optical axis) and
    tall enough for the part above it.  Unstated values (indices, absorption) as in the
    256^3 workload."""
    h = 0.216
    top = float(fin_bottoms_mm(n_fins)[-1]) + FIN_THICK_MM + 1.0
    nz = 2 * int(math.ceil(top / h))
    return Workload(name=f"fins{n_fins}_nontelecentric_{nz}z", nx=112, ny=112, nz=nz, voxel_mm=h,
                    nu=112, nv=nz, pixel_u_mm=h, pixel_v_mm=h, n_angles=360, pupil_mm=99.5, f_number=INF,
                    pupil_pattern="chief", rays_per_pixel=1, r_inner_mm=11.8, wall_mm=0.7, n_outside=1.0,
                    n_glass=1.47, n_resin=1.50, mu_per_mm=0.03, target=f"fins{n_fins}", osmo_iters=40)


def etendue_workload(iris_diameter_mm: float = 16.0, rays: str = "hex13") -> Workload:
    """The telecentric printer of Sec. 2.6.2 (the parameterised 4f relay of
    `telecentric_relay` with the given iris; vial OD 8 / ID 6.6 mm) on a 0.05 mm grid
    (coarser than the paper's 0.0432 mm) 3.2 mm tall, 360 angles.  rays: "hex13" (13
    rays per pixel, the paper's etendue model) or "chief" (one ray, zero etendue)."""
    n = 13 if rays == "hex13" else 1
    return Workload(name=f"telecentric_iris{iris_diameter_mm:g}_{rays}", nx=136, ny=136, nz=64, voxel_mm=0.05,
                    nu=136, nv=64, pixel_u_mm=0.05, pixel_v_mm=0.05, n_angles=360, pupil_mm=INF, f_number=INF,
                    pupil_pattern=rays, rays_per_pixel=n, r_inner_mm=3.3, wall_mm=0.7, n_outside=1.0,
                    n_glass=1.47, n_resin=1.50, mu_per_mm=0.05, target="csg_shells", osmo_iters=20,
                    lens=telecentric_relay(iris_diameter_mm=iris_diameter_mm))


def radon_workload(w: Workload) -> Workload:
    """The printer the Radon method assumes (Sec. 2.3): parallel chief rays (telecentric,
    zero etendue), no refraction (all indices 1) and no attenuation, on w's grid, pixels
    and angles -- the geometry in which the ray-traced projection is the per-slice
    parallel-beam Radon transform."""
    return replace(w, name=w.name + "_radon", pupil_mm=INF, f_number=INF, pupil_pattern="chief",
                   rays_per_pixel=1, n_outside=1.0, n_glass=1.0, n_resin=1.0, mu_per_mm=0.0)


def default_angles(n_angles: int) -> np.ndarray:
    """theta_k = 2*pi*k/N (a full turn in equal steps, Sec. 2.5)."""
    return 2.0 * np.pi * np.arange(n_angles, dtype=np.float64) / n_angles


# ----------------------------------------------------------------------------------
# binary targets (float32 {0,1}, layout [nz][ny][nx], voxel centres at (i-(N-1)/2)*h)
# ----------------------------------------------------------------------------------
def voxel_centres(w: Workload):
    h = w.voxel_mm
    x = (np.arange(w.nx) - (w.nx - 1) / 2.0) * h
    y = (np.arange(w.ny) - (w.ny - 1) / 2.0) * h
    z = (np.arange(w.nz) - (w.nz - 1) / 2.0) * h
    return np.meshgrid(z, y, x, indexing="ij")  # Z, Y, X each [nz][ny][nx]


def reach_radius(w: Workload, margin_mm: float = 0.3) -> float:
    """Radius inside which every direction is available to some ray (target placement)."""
    r_o = w.r_inner_mm + w.wall_mm
    b_max = min(w.nu * w.pixel_u_mm / 2.0, r_o, w.n_glass * w.r_inner_mm / w.n_outside)
    return b_max * w.n_outside / w.n_resin - margin_mm


def _sphere(Z, Y, X, c, r):
    return (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r


def _box(Z, Y, X, c, half):
    return (np.abs(X - c[0]) <= half[0]) & (np.abs(Y - c[1]) <= half[1]) & (np.abs(Z - c[2]) <= half[2])


def _torus(Z, Y, X, c, axis, R, r):
    px, py, pz = X - c[0], Y - c[1], Z - c[2]
    along = px * axis[0] + py * axis[1] + pz * axis[2]
    radial2 = np.maximum(px * px + py * py + pz * pz - along * along, 0.0)
    return (np.sqrt(radial2) - R) ** 2 + along * along <= r * r


def _rand_axis(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _rand_centre(rng, w: Workload, extent: float, reach: float):
    """Centre such that a primitive of bounding radius `extent` stays in reach and grid."""
    rmax = max(reach - extent, 0.0)
    rad = rmax * math.sqrt(rng.random())
    phi = 2.0 * math.pi * rng.random()
    zmax = max(w.nz * w.voxel_mm / 2.0 - extent - 2.0 * w.voxel_mm, 0.0)
    return (rad * math.cos(phi), rad * math.sin(phi), rng.uniform(-zmax, zmax))


def _axis(n: int, h: float, i0: int = 0, i1: Optional[int] = None) -> np.ndarray:
    """Voxel-centre coordinates (i - (n-1)/2) h of indices i0 .. i1-1 (the values
    voxel_centres gives, computed the same way)."""
    return (np.arange(i0, n if i1 is None else i1) - (n - 1) / 2.0) * h


class _Grid:
    """Broadcastable voxel-centre coordinates and bounded sub-box evaluation of a primitive:
    a primitive whose points all lie within `extent` mm of its centre is evaluated only on
    the index box that covers that ball, with coordinates computed exactly as on the full
    grid, so the result equals a full-grid evaluation."""

    def __init__(self, w: Workload):
        self.w = w
        self.n = (w.nx, w.ny, w.nz)
        self.h = w.voxel_mm
        self.X = _axis(w.nx, self.h)[None, None, :]
        self.Y = _axis(w.ny, self.h)[None, :, None]
        self.Z = _axis(w.nz, self.h)[:, None, None]

    def _range(self, ax: int, c: float, extent: float):
        n = self.n[ax]
        lo = int(math.floor((c - extent) / self.h + (n - 1) / 2.0)) - 1
        hi = int(math.ceil((c + extent) / self.h + (n - 1) / 2.0)) + 2
        return max(lo, 0), min(hi, n)

    def apply(self, m: np.ndarray, fn, c, extent: float, union: bool = True):
        """m |= fn(Z, Y, X) (union) or m &= ~fn(Z, Y, X) inside the primitive's box."""
        (x0, x1), (y0, y1), (z0, z1) = (self._range(a, c[a], extent) for a in range(3))
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            return
        h = self.h
        Z = _axis(self.n[2], h, z0, z1)[:, None, None]
        Y = _axis(self.n[1], h, y0, y1)[None, :, None]
        X = _axis(self.n[0], h, x0, x1)[None, None, :]
        p = fn(Z, Y, X)
        if union:
            m[z0:z1, y0:y1, x0:x1] |= p
        else:
            m[z0:z1, y0:y1, x0:x1] &= ~p


def make_target(w: Workload, kind: Optional[str] = None, seed: Optional[int] = None) -> np.ndarray:
    kind = kind or w.target
    seed = w.seed if seed is None else seed
    rng = np.random.default_rng(seed + 1000)
    G = _Grid(w)
    Z, Y, X = G.Z, G.Y, G.X          # broadcastable [nz,1,1], [1,ny,1], [1,1,nx]
    reach = reach_radius(w)
    m = np.zeros(w.vol_shape, dtype=bool)
    if kind == "sphere_cube":
        # sphere r = 4 mm centred (0,0,-1.5) united with a 3 mm cube centred (1,1,3.5)
        m |= _sphere(Z, Y, X, (0.0, 0.0, -1.5), 4.0) | _box(Z, Y, X, (1.0, 1.0, 3.5), (1.5, 1.5, 1.5))
    elif kind == "spheres_tori12":
        for k in range(12):
            if k % 2 == 0:
                r = rng.uniform(1.0, 5.0)
                c = _rand_centre(rng, w, r, reach)
                G.apply(m, lambda Z, Y, X, c=c, r=r: _sphere(Z, Y, X, c, r), c, r)
            else:
                R = rng.uniform(1.0, 5.0)
                r = rng.uniform(0.35, 0.3 * R + 0.35)
                c = _rand_centre(rng, w, R + r, reach)
                ax = _rand_axis(rng)
                G.apply(m, lambda Z, Y, X, c=c, ax=ax, R=R, r=r: _torus(Z, Y, X, c, ax, R, r), c, R + r)
    elif kind == "strut_lattice":
        cell, beam = 4.0, 0.5
        off = rng.uniform(0.0, cell, size=3)
        keep = 0.75
        # beams along x, y and z through the lattice points; each beam family keeps a
        # seeded random subset of the lines
        gx = np.mod(X - off[0] + cell / 2, cell) - cell / 2
        gy = np.mod(Y - off[1] + cell / 2, cell) - cell / 2
        gz = np.mod(Z - off[2] + cell / 2, cell) - cell / 2
        ix = np.floor((X - off[0] + cell / 2) / cell).astype(np.int64)
        iy = np.floor((Y - off[1] + cell / 2) / cell).astype(np.int64)
        iz = np.floor((Z - off[2] + cell / 2) / cell).astype(np.int64)
        salt = rng.integers(1, 2**31 - 1, size=3)

        def keep_line(a, b, s):
            hsh = (a * 73856093) ^ (b * 19349663) ^ s
            return (hsh % 1000) < int(keep * 1000)

        hb = beam / 2
        m |= (np.abs(gy) <= hb) & (np.abs(gz) <= hb) & keep_line(iy, iz, salt[0])
        m |= (np.abs(gx) <= hb) & (np.abs(gz) <= hb) & keep_line(ix, iz, salt[1])
        m |= (np.abs(gx) <= hb) & (np.abs(gy) <= hb) & keep_line(ix, iy, salt[2])
        m &= X * X + Y * Y <= min(10.0, reach) ** 2
        zlim = w.nz * w.voxel_mm / 2.0 - 1.0
        m &= np.abs(Z) <= zlim
    elif kind in ("csg", "csg_shells"):
        n_prim = 40 if kind == "csg_shells" else int(rng.integers(3, 7))
        scale = min(reach, w.nz * w.voxel_mm / 2.0)
        for k in range(n_prim):
            t = rng.integers(0, 3)
            if t == 0:
                r = rng.uniform(0.12, 0.35) * scale
                c = _rand_centre(rng, w, r, reach)
                fn, ext = (lambda Z, Y, X, c=c, r=r: _sphere(Z, Y, X, c, r)), r
            elif t == 1:
                half = rng.uniform(0.08, 0.3, size=3) * scale
                ext = float(np.linalg.norm(half))
                c = _rand_centre(rng, w, ext, reach)
                fn = lambda Z, Y, X, c=c, half=half: _box(Z, Y, X, c, half)  # noqa: E731
            else:
                R = rng.uniform(0.15, 0.35) * scale
                r = rng.uniform(0.25, 0.5) * R
                c = _rand_centre(rng, w, R + r, reach)
                ax = _rand_axis(rng)
                fn, ext = (lambda Z, Y, X, c=c, ax=ax, R=R, r=r: _torus(Z, Y, X, c, ax, R, r)), R + r
            if kind == "csg_shells" and k % 4 == 3 and t == 0:
                # thin-walled shell of 0.3 mm
                ri = max(r - 0.3, 0.0)
                fn = lambda Z, Y, X, c=c, r=r, ri=ri: _sphere(Z, Y, X, c, r) & ~_sphere(Z, Y, X, c, ri)  # noqa: E731
            G.apply(m, fn, c, ext, union=not (k > 0 and rng.random() < 0.25))
        m &= X * X + Y * Y <= reach * reach
    elif kind.startswith("fins"):
        n_fins = int(kind[4:])
        hx = FIN_HALF_MM
        zt = float(fin_bottoms_mm(n_fins)[-1]) + FIN_THICK_MM
        m |= _box(Z, Y, X, (0.0, 0.0, FIN_BASE_MM / 2), (hx, hx, FIN_BASE_MM / 2))           # base
        m |= _box(Z, Y, X, (0.0, hx - 0.5, zt / 2), (hx, 0.5, zt / 2))                      # spine
        for zb in fin_bottoms_mm(n_fins):
            m |= _box(Z, Y, X, (0.0, 0.0, zb + FIN_THICK_MM / 2), (hx, hx, FIN_THICK_MM / 2))
    else:
        raise ValueError(f"unknown target {kind!r}")
    return m.astype(np.float32)


def random_volume(w: Workload, seed: int = 1) -> np.ndarray:
    return np.random.default_rng(seed).random(w.vol_shape, dtype=np.float32)


def random_projections(w: Workload, seed: int = 2) -> np.ndarray:
    return np.random.default_rng(seed).random(w.proj_shape, dtype=np.float32)


def sparse_projections(w: Workload, n_nonzero: int, seed: int = 3) -> np.ndarray:
    """Projections that are zero except at n_nonzero seeded pixels (values in [0.5, 1.5))."""
    rng = np.random.default_rng(seed)
    g = np.zeros(w.proj_shape, dtype=np.float32)
    flat = rng.choice(g.size, size=n_nonzero, replace=False)
    g.flat[flat] = 0.5 + rng.random(n_nonzero, dtype=np.float32)
    return g
