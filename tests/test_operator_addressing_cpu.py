"""CPU emulation of the operator kernels' memory addressing (the tiled traversal shared by
the projection and the dose, paper_2211_03516_gb300/csrc/operators.cu).

For sampled pixel tiles of the workloads at several angles, every ray's table entry is
built from the FP64 oracle's trace (the quantities the ray-table kernel stores: entry
point and step in voxels, direction, the sample range whose footprint reaches the grid in
z), and the kernel's integer and FP32 steps are repeated exactly as written: Q32.32 start
and step per angle, the trimming of the sample range, chunk and half-chunk sample ranges,
Q9.23 anchors and steps, the block's footprint box, the fit and in-grid decisions with the
retry as two halves, the backward walk inside a box and the exact-position walk on global
memory.  Checked: every staged row lies inside the padded grid, every sample of a boxed
chunk reads or updates its 8 corners inside the box, every sample walked on global memory
has its 8 corners inside the padded grid, and each ray's samples are covered exactly once.
Needs no GPU; the table comes from the oracle, so it checks the kernel's addressing design
on the workloads' real geometry, not the ray-table kernel's own rounding.
"""
import math
import os
import re

import numpy as np
import pytest

from oracle import vam_oracle as O
from paper_2211_03516_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_03516_gb300", "csrc")

f32 = np.float32


def _constants():
    """Tiling constants as the kernels compile them."""
    src = open(os.path.join(CSRC, "internal.cuh")).read() + open(os.path.join(CSRC, "operators.cu")).read()
    out = {}
    for name in ("kTileU", "kTileV", "kChunkVox", "kBoxFloats", "kMaxBoxExtent"):
        m = re.search(r"constexpr int %s = ([0-9 *]+);" % name, src)
        assert m, name
        out[name] = int(eval(m.group(1)))   # plain integer products such as 18 * 1024
    return out


C = _constants()


class Padded:
    """The padded scratch volume and the launch constants of make_projector."""

    def __init__(self, w):
        self.px = ((w.nx + 2 + 3) // 4) * 4
        self.py = w.ny + 2
        self.pz = w.nz + 2
        self.cx = 0.5 * (w.nx - 1) + 1.0
        self.cy = 0.5 * (w.ny - 1) + 1.0
        self.cz = 0.5 * (w.nz - 1) + 1.0
        self.y0 = f32(-w.r_inner_mm / w.voxel_mm - 1.0)


def table_entry(w, pupil, u, v, a):
    """(A, B, jlo, jhi) of one ray as the ray-table kernel stores it, or None (no resin)."""
    r = O.trace(w, pupil, u, v, a)
    if r["status"] != 2:
        return None
    h = w.voxel_mm
    e, d = r["e"], r["d2"]
    K = int(r["k"])
    delta = r["ell"] / K
    zc = 0.5 * (w.nz - 1)
    j = np.arange(K)
    qz = (e[2] + ((j + 0.5) * delta) * d[2]) / h + zc
    inside = np.nonzero((qz > -1.0) & (qz < w.nz))[0]
    if inside.size == 0:
        return None
    A = (e[0] / h, e[1] / h, e[2] / h, delta / h)
    B = (d[0], d[1], d[2])
    return A, B, int(inside[0]), int(inside[-1]) + 1


def q32(x):
    return int(np.rint(x * 4294967296.0))


class Ray:
    """ray_begin: the Q32.32 start and step at one angle, the FP32 chunking values, the
    Q9.23 step and the trimmed sample range [jlo, jhi) (empty when no sample remains)."""

    def __init__(self, G, entry, cs):
        A, B, jlo, jhi = entry
        c, s = cs
        ex, ey, dl = A[0], A[1], A[3]
        stx = (c * B[0] - s * B[1]) * dl
        sty = (s * B[0] + c * B[1]) * dl
        stz = B[2] * dl
        self.q0 = [q32(G.cx + (c * ex - s * ey) + 0.5 * stx), q32(G.cy + (s * ex + c * ey) + 0.5 * sty),
                   q32(G.cz + A[2] + 0.5 * stz)]
        self.s = [q32(stx), q32(sty), q32(stz)]
        self.d23 = [(si + 256) >> 9 for si in self.s]
        self.ey = f32(A[1])
        self.dy = f32(A[3] * B[1])
        self.inv_dy = f32(1.0) / self.dy if self.dy != 0 else f32(np.inf)
        zmax = (G.pz - 1) << 32

        def z_in(j):
            qz = self.q0[2] + j * self.s[2]
            return 0 <= qz < zmax

        for _ in range(4):
            if jlo < jhi and not z_in(jlo):
                jlo += 1
        for _ in range(4):
            if jlo < jhi and not z_in(jhi - 1):
                jhi -= 1
        if jlo < jhi and not (z_in(jlo) and z_in(jhi - 1)):
            jhi = jlo
        self.jlo, self.jhi = jlo, jhi

    def y_at(self, j):
        # fmaf((float)j + 0.5f, dy, ey): one rounding of the exact product-sum
        return f32(float(f32(j + 0.5)) * float(self.dy) + float(self.ey))


MIN_DY = f32(1e-4)


def chunk_of(G, R, j):
    return int(math.floor(f32(f32(R.y_at(j) - G.y0) * f32(1.0 / C["kChunkVox"]))))


def half_start(G, R, h):
    yc = f32(G.y0 + f32(h * (C["kChunkVox"] // 2)))
    j = math.ceil(f32(f32(f32(yc - R.ey) * R.inv_dy) - f32(0.5)))
    return int(min(max(j, R.jlo), R.jhi))


def range_samples(G, R, h0, h1, cmin, cmax):
    if not (R.dy > MIN_DY):
        return (R.jlo if h0 == 2 * cmin else R.jhi), R.jhi
    jl = R.jlo if h0 == 2 * cmin else half_start(G, R, h0)
    jh = R.jhi if h1 == 2 * cmax + 2 else half_start(G, R, h1)
    return jl, jh


def emulate_block(G, rays):
    """One block's traversal of one aperture sample (rays: the active Ray objects of its
    pixels).  Returns (boxed samples, global samples); asserts every access in bounds."""
    if not rays:
        return 0, 0
    cf = [chunk_of(G, R, R.jlo) for R in rays]
    cl = [max(chunk_of(G, R, R.jhi - 1) if R.dy > MIN_DY else c0, c0) for R, c0 in zip(rays, cf)]
    cmin, cmax = min(cf), max(cl)
    covered = [np.zeros(R.jhi - R.jlo, np.int32) for R in rays]
    n_box = n_glob = 0
    for c in range(cmin, cmax + 1):
        nsplit, part = 1, 0
        while part < nsplit:
            h0 = 2 * c + part * (2 // nsplit)
            h1 = h0 + 2 // nsplit
            ranges, lo, hi = [], [math.inf] * 3, [-math.inf] * 3
            for R in rays:
                jl, jh = range_samples(G, R, h0, h1, cmin, cmax)
                an = None
                if jl < jh:
                    an = [(R.q0[d] + (jh - 1) * R.s[d]) >> 9 for d in range(3)]
                    n = jh - 1 - jl
                    for d in range(3):
                        c0, c1 = an[d] >> 23, (an[d] - n * R.d23[d]) >> 23
                        lo[d] = min(lo[d], c0, c1)
                        hi[d] = max(hi[d], max(c0, c1) + 1)
                ranges.append((jl, jh, an))
            part += 1
            if hi[0] == -math.inf:
                continue
            bx0, by0, bz0 = lo[0] & ~3, lo[1], lo[2]
            hx, hy, hz = hi
            ex = ((hx + 4) & ~3) - bx0
            ey, ez = hy + 1 - by0, hz + 1 - bz0
            sx = ex + 1
            sxy = sx * (ey | 1)
            in_grid = lo[0] >= 0 and by0 >= 0 and bz0 >= 0 and hx <= G.px - 1 and hy <= G.py - 1 and hz <= G.pz - 1
            fits = (sxy * ez <= C["kBoxFloats"] and ex <= C["kMaxBoxExtent"] and ey <= C["kMaxBoxExtent"]
                    and ez <= C["kMaxBoxExtent"])
            if not fits and nsplit == 1 and in_grid:
                nsplit, part = 2, 0          # retried as two halves
                continue
            for R, cov, (jl, jh, an) in zip(rays, covered, ranges):
                if jl >= jh:
                    continue
                cov[jl - R.jlo:jh - R.jlo] += 1
                j = np.arange(jl, jh, dtype=np.int64)
                if fits and in_grid:
                    # staged rows: planes bz0..bz0+ez-1, rows by0..by0+ey-1, x bx0..bx0+ex-1
                    assert bz0 + ez - 1 <= G.pz - 1 and by0 + ey - 1 <= G.py - 1 and bx0 + ex - 1 <= G.px - 1
                    assert ex % 4 == 0 and bx0 % 4 == 0
                    ext = (ex, ey, ez)
                    lin = np.zeros(j.size, np.int64)
                    for d, (o, stride) in enumerate(((bx0, 1), (by0, sx), (bz0, sxy))):
                        q = (an[d] - (o << 23)) - (jh - 1 - j) * R.d23[d]
                        assert 0 <= q.min() and q.max() < (1 << 31)          # a 32-bit Q9.23 offset
                        cell = q >> 23
                        assert cell.min() >= 0 and cell.max() + 1 <= ext[d] - 1
                        lin += cell * stride
                    assert lin.max() + sxy + sx + 1 < sxy * ez
                    n_box += j.size
                else:
                    for d, p in enumerate((G.px, G.py, G.pz)):
                        cell = (R.q0[d] + j * R.s[d]) >> 32
                        assert cell.min() >= 0 and cell.max() + 1 <= p - 1
                    n_glob += j.size
    for cov in covered:
        assert (cov == 1).all()                      # each sample in exactly one chunk
    return n_box, n_glob


def tiles_for(w, n_tiles, rng):
    """Pixel tiles (u0, v0): the centre, the ragged corner, and random others."""
    nut = (w.nu + C["kTileU"] - 1) // C["kTileU"]
    nvt = (w.nv + C["kTileV"] - 1) // C["kTileV"]
    tiles = {(nut // 2, nvt // 2), (nut - 1, nvt - 1), (0, 0)}
    while len(tiles) < n_tiles:
        tiles.add((int(rng.integers(nut)), int(rng.integers(nvt))))
    return [(tu * C["kTileU"], tv * C["kTileV"]) for tu, tv in sorted(tiles)]


def run_workload(w, angles, n_tiles, seed=0, min_box_fraction=0.0):
    pupil = I.workload_pupil(w)
    G = Padded(w)
    rng = np.random.default_rng(seed)
    cache = {}
    n_box = n_glob = 0
    for (u0, v0) in tiles_for(w, n_tiles, rng):
        for k in angles:
            th = 2.0 * math.pi * k / w.n_angles
            cs = (math.cos(th), math.sin(th))
            for a in range(w.rays_per_pixel):
                rays = []
                for u in range(u0, min(u0 + C["kTileU"], w.nu)):
                    for v in range(v0, min(v0 + C["kTileV"], w.nv)):
                        key = (u, v, a)
                        if key not in cache:
                            cache[key] = table_entry(w, pupil, u, v, a)
                        if cache[key] is None:
                            continue
                        R = Ray(G, cache[key], cs)
                        if R.jlo < R.jhi:
                            rays.append(R)
                b, g = emulate_block(G, rays)
                n_box += b
                n_glob += g
    assert n_box + n_glob > 0
    assert n_box / (n_box + n_glob) >= min_box_fraction
    return n_box, n_glob


SMALL = {
    "tiny": (I.TINY, (0, 11, 23, 45, 67)),
    "refracting_ragged": (I.TINY.scaled(nx=33, ny=34, nz=23, voxel_mm=0.4, nu=37, nv=23, pixel_u_mm=0.38,
                                        pixel_v_mm=0.41, n_angles=10, f_number=3.5, pupil_pattern="sunflower",
                                        rays_per_pixel=4, pupil_mm=60.0), (0, 1, 3, 7)),
    "lens_train": (I.TINY.scaled(nx=33, ny=34, nz=23, voxel_mm=0.4, nu=37, nv=23, pixel_u_mm=0.38,
                                 pixel_v_mm=0.41, n_angles=10, f_number=3.5, pupil_mm=60.0,
                                 lens=I.telecentric_relay(), pupil_pattern="hex13", rays_per_pixel=13), (0, 2, 5)),
    "fins18": (I.fins_workload(18).scaled(n_angles=24), (0, 3, 5, 17)),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_addressing_in_bounds_small_workloads(name):
    w, angles = SMALL[name]
    run_workload(w, angles, n_tiles=4)


# The full-size workloads: a few tiles at angles along the axes and the diagonals, where
# the footprint boxes are largest.  Most samples must run from shared memory.
LARGE = {
    "mid_256cube_stratified_per_pixel": (I.MID, (0, 45, 23), 0.98),
    "tall_384x384x512": (I.WORKLOADS["tall_384x384x512_720ang_8rays"], (0, 90, 157), 0.99),
    "large_768x768x1024": (I.WORKLOADS["large_768x768x1024_1000ang_4rays"], (0, 125, 63, 311), 0.99),
}


@pytest.mark.parametrize("name", list(LARGE))
def test_addressing_in_bounds_full_size_tiles(name):
    w, angles, min_box = LARGE[name]
    run_workload(w, angles, n_tiles=3, seed=1, min_box_fraction=min_box)
