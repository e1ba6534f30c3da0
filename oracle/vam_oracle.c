/*
 * FP64 CPU oracle for the 3D ray-traced tomographic projection and dose operators of
 * "Versatile volumetric additive manufacturing with 3D ray tracing" (Webber et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this file:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header or constant with the CUDA library; both are written from
 * the paper's description.
 *
 * What is computed, in the paper's order (every loop is plain and sequential):
 *   Sec. 2.1  ray generation: for each pixel, rays leave points of the aperture stop
 *             and converge on the pixel's image point in the best-focus plane; the
 *             chief ray leaves the centre of the stop.  Vector Snell's law at each
 *             cylinder surface (air/glass, glass/resin); tracing stops at the inner
 *             wall on the far side of the vial.
 *   Sec. 2.2  anti-aliasing: each sample on the ray interacts with the neighbouring
 *             voxels with weight (1-dx)(1-dy)(1-dz) (trilinear weights).
 *   Sec. 2.4  projection: pixel value = sum over its rays of the weighted voxel values
 *             along the ray.  With the Beer-Lambert and Fresnel factors of Sec. 2.5 it
 *             is the exact transpose (adjoint) of the dose operator below.
 *   Sec. 2.5  dose: every sample adds pixel intensity x anti-aliasing weight x Fresnel
 *             transmission (unpolarised) x Beer-Lambert transmission to its voxels.
 *             Repeated for all rays of all pixels and all rotation angles.
 * Readings where the paper is silent: samples are midpoints s_j = (j+1/2) ell/K with
 * K = ceil(ell/ds) (the per-ray step makes the sample sum of a unit field equal to the
 * chord length); voxel centres sit at (i-(N-1)/2) h; corners outside the grid count
 * as zero; Fresnel losses at both the outer and inner surfaces; the vial rotates by
 * theta_k about z, applied to the traced path as x' = R(theta_k) x.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t nx, ny, nz;
    double h;               /* voxel pitch, mm */
    int32_t nu, nv;
    double pu, pv;          /* pixel pitch in the best-focus plane y = 0, mm */
    double pupil;           /* distance of the aperture stop from the axis; INFINITY = telecentric */
    double fnum;            /* f-number: stop diameter = pupil / fnum; INFINITY = chief ray only */
    int32_t m;              /* rays per pixel */
    const double *pupil_xy; /* m points (xi, eta) in the unit disk */
    double r_in, wall;      /* vial inner radius and wall thickness, mm */
    double n_out, n_glass, n_resin;
    double mu;              /* absorption coefficient, 1/mm */
    int32_t n_angles;
    const double *angles;   /* radians */
    double step_vox;        /* nominal sample spacing in voxels */
    int32_t unattenuated;   /* projection only: weight delta / M, no Fresnel or Beer-Lambert (Sec. 2.4 as printed) */
    /* Optional lens train between the pixel array and the vial (Sec. 2.1: rays refract at
     * every optical element; Sec. 2.6.2: two plano-spherical lenses and an iris).  When
     * n_surf > 0 it replaces the pupil model: pixel (u,v) sits at Q_uv / mag in the plane
     * y = obj_y, aperture sample (xi, eta) leaves it with direction proportional to
     * (xi r_s / aim, 1, eta r_s / aim) (r_s the stop radius), and the ray is refracted by
     * Snell's law at each surface (transmission 1: coated lenses), blocked by any clear
     * aperture it falls outside of, and handed to the vial in air. */
    int32_t n_surf;
    const double *surf;     /* n_surf x 5: vertex y, radius (INFINITY = plane; centre at y + radius),
                               index after, clear semi-aperture, stop flag */
    double obj_y, mag, aim;
    /* Aperture-stop samples generated here instead of read from pupil_xy (Sec. 2.1: rays
     * leave points of the stop; the paper fills it hexagonally).  0 = the list pupil_xy;
     * 1 = chief ray only; 2 = n x n stratified jitter (m = n^2) mapped to the disk by the
     * concentric map; 3 = golden-angle sunflower; 4 = hexagonal filling, 13 rays.
     * per_pixel: the jitter draws depend on the pixel (u, v), else they are shared by every
     * pixel.  Jitter numbers come from splitmix64 of seed ^ key(u, v, a, c). */
    int32_t aperture;
    int32_t per_pixel;
    uint64_t seed;
} orc_geom;

typedef struct {
    int32_t status;         /* 2 reaches the resin, 1 only crosses the wall, 0 misses, -1 total internal reflection */
    int32_t k;              /* samples on the in-resin segment */
    double origin[3], d0[3];/* ray leaving the projector */
    double p1[3], d1[3];    /* outer-surface hit, direction in the glass */
    double e[3], d2[3];     /* resin entry point, direction in the resin */
    double exit[3];         /* far-side inner-wall point */
    double ell;             /* in-resin length, mm */
    double t1, t2;          /* Fresnel transmissions at the outer and inner surface */
} orc_ray;

/* Intersections of the line o + t d with the infinite cylinder x^2 + y^2 = r^2.
 * Returns 0 when the line misses it (or runs parallel to the axis). */
static int cylinder_roots(const double o[3], const double d[3], double r, double *t_near, double *t_far)
{
    double a = d[0] * d[0] + d[1] * d[1];
    double b = 2.0 * (o[0] * d[0] + o[1] * d[1]);
    double c = o[0] * o[0] + o[1] * o[1] - r * r;
    if (a <= 0.0) return 0;
    double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) return 0;
    double q = -0.5 * (b + (b >= 0.0 ? sqrt(disc) : -sqrt(disc)));
    if (q == 0.0) return 0;
    double r1 = q / a, r2 = c / q;
    *t_near = r1 < r2 ? r1 : r2;
    *t_far = r1 < r2 ? r2 : r1;
    return 1;
}

/* Vector form of Snell's law at a cylinder surface point p (radius r) for unit
 * direction d going from index n1 to n2.  Writes the refracted direction and the
 * unpolarised Fresnel transmission.  Returns 0 on total internal reflection. */
static int refract(const double p[3], double r, const double d[3], double n1, double n2,
                   double out[3], double *trans)
{
    double n[3] = {p[0] / r, p[1] / r, 0.0};
    double cn = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
    if (cn > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; cn = -cn; }
    double c1 = -cn;                         /* cosine of the incidence angle */
    double eta = n1 / n2;
    double k = 1.0 - eta * eta * (1.0 - c1 * c1);
    if (k < 0.0) return 0;
    double c2 = sqrt(k);                     /* cosine of the refraction angle */
    for (int i = 0; i < 3; ++i) out[i] = eta * d[i] + (eta * c1 - c2) * n[i];
    double rs = (n1 * c1 - n2 * c2) / (n1 * c1 + n2 * c2);
    double rp = (n1 * c2 - n2 * c1) / (n1 * c2 + n2 * c1);
    *trans = 1.0 - 0.5 * (rs * rs + rp * rp);
    return 1;
}

/* Snell's law in vector form for a unit normal nrm (either orientation) and unit
 * direction d, index n1 -> n2.  Returns 0 on total internal reflection. */
static int refract_normal(const double nrm[3], const double d[3], double n1, double n2, double out[3])
{
    double n[3] = {nrm[0], nrm[1], nrm[2]};
    double cn = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
    if (cn > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; cn = -cn; }
    double c1 = -cn, eta = n1 / n2;
    double k = 1.0 - eta * eta * (1.0 - c1 * c1);
    if (k < 0.0) return 0;
    double c2 = sqrt(k);
    for (int i = 0; i < 3; ++i) out[i] = eta * d[i] + (eta * c1 - c2) * n[i];
    return 1;
}

/* Carry the ray (o, d) through the lens train; on return o is its point on the last
 * surface and d its direction in the air behind it.  Returns 0 when a surface is missed
 * or a clear aperture blocks the ray (or on total internal reflection). */
int orc_lens_train(const orc_geom *g, double o[3], double d[3])
{
    double n_cur = g->n_out;
    for (int s = 0; s < g->n_surf; ++s) {
        const double *S = g->surf + 5 * s;
        double yv = S[0], R = S[1], n2 = S[2], clear = S[3];
        int stop = S[4] != 0.0;
        double t, p[3], nrm[3];
        if (isinf(R)) {
            if (d[1] == 0.0) return 0;
            t = (yv - o[1]) / d[1];
        } else {
            /* sphere of radius |R| centred at (0, yv + R, 0): the root on the vertex side */
            double c[3] = {0.0, yv + R, 0.0};
            double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
            double b = d[0] * oc[0] + d[1] * oc[1] + d[2] * oc[2];
            double cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - R * R;
            double disc = b * b - cc;
            if (disc < 0.0) return 0;
            double sq = sqrt(disc), roots[2] = {-b - sq, -b + sq};
            t = -1.0;
            for (int k = 0; k < 2 && t < 0.0; ++k) {
                double py = o[1] + roots[k] * d[1];
                if (roots[k] > 0.0 && (py - c[1]) * (yv - c[1]) > 0.0) t = roots[k];
            }
        }
        if (!(t > 0.0)) return 0;
        for (int i = 0; i < 3; ++i) p[i] = o[i] + t * d[i];
        if (p[0] * p[0] + p[2] * p[2] > clear * clear) return 0;
        if (!stop) {
            if (isinf(R)) { nrm[0] = 0.0; nrm[1] = 1.0; nrm[2] = 0.0; }
            else { nrm[0] = p[0] / R; nrm[1] = (p[1] - (yv + R)) / R; nrm[2] = p[2] / R; }
            double out[3];
            if (!refract_normal(nrm, d, n_cur, n2, out)) return 0;
            for (int i = 0; i < 3; ++i) d[i] = out[i];
        }
        for (int i = 0; i < 3; ++i) o[i] = p[i];
        n_cur = n2;
    }
    return 1;
}

/* splitmix64 (Steele, Lea and Flood 2014; Vigna's public-domain form): one step of the
 * generator from state x, i.e. the Weyl increment followed by the variant-13 finaliser. */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

/* Jitter number in [0, 1) for pixel (u, v), aperture sample a and component c (0 or 1):
 * the top 53 bits of splitmix64(seed ^ key), key = u + 2^20 v + 2^40 a + 2^56 c. */
double orc_jitter(uint64_t seed, int32_t u, int32_t v, int32_t a, int32_t c)
{
    uint64_t key = (uint64_t)(uint32_t)u | ((uint64_t)(uint32_t)v << 20) | ((uint64_t)(uint32_t)a << 40) |
                   ((uint64_t)(uint32_t)c << 56);
    return (double)(splitmix64(seed ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

/* Shirley and Chiu's concentric map of the square [-1,1]^2 onto the unit disk: squares
 * centred on the origin go to circles, the four triangular sectors between the diagonals
 * to the four quarter disks, preserving area fractions. */
static void concentric(double p, double q, double out[2])
{
    double r, phi;
    if (p == 0.0 && q == 0.0) { out[0] = 0.0; out[1] = 0.0; return; }
    if (fabs(p) > fabs(q)) { r = p; phi = (ORC_PI / 4.0) * (q / p); }
    else { r = q; phi = ORC_PI / 2.0 - (ORC_PI / 4.0) * (p / q); }
    out[0] = r * cos(phi);
    out[1] = r * sin(phi);
}

/* Aperture-stop point (xi, eta) in the unit disk of aperture sample a of pixel (u, v). */
void orc_aperture_point(const orc_geom *g, int32_t u, int32_t v, int32_t a, double out[2])
{
    int32_t pu = g->per_pixel ? u : 0, pv = g->per_pixel ? v : 0;
    out[0] = 0.0; out[1] = 0.0;
    if (g->aperture == 0) { out[0] = g->pupil_xy[2 * a]; out[1] = g->pupil_xy[2 * a + 1]; return; }
    if (g->aperture == 1) return;                              /* the chief ray: the stop's centre */
    if (g->aperture == 2) {
        /* n x n strata of [-1,1]^2, one jittered point in stratum (i, k), a = i n + k */
        int32_t n = (int32_t)floor(sqrt((double)g->m) + 0.5);
        int32_t i = a / n, k = a % n;
        double p = 2.0 * (i + orc_jitter(g->seed, pu, pv, a, 0)) / n - 1.0;
        double q = 2.0 * (k + orc_jitter(g->seed, pu, pv, a, 1)) / n - 1.0;
        concentric(p, q, out);
        return;
    }
    if (g->aperture == 3) {
        /* sunflower: radius sqrt((a + 1/2)/m), azimuth a times the golden angle, the whole
         * pattern turned by 2 pi times one jitter number of the pixel */
        double golden = ORC_PI * (3.0 - sqrt(5.0));
        double r = sqrt((a + 0.5) / g->m);
        double phi = a * golden + 2.0 * ORC_PI * orc_jitter(g->seed, pu, pv, 0, 0);
        out[0] = r * cos(phi);
        out[1] = r * sin(phi);
        return;
    }
    /* hexagonal filling of the stop (Sec. 2.1) read as the points of a hexagonal lattice of
     * spacing 1/2 inside the unit disk: the centre, 6 at distance 1/2 (azimuths 0, 60, ...,
     * 300 degrees) and 6 at distance sqrt(3)/2 (30, 90, ..., 330 degrees) */
    if (a == 0) return;
    if (a <= 6) {
        double t = (a - 1) * ORC_PI / 3.0;
        out[0] = 0.5 * cos(t); out[1] = 0.5 * sin(t);
        return;
    }
    double t = ORC_PI / 6.0 + (a - 7) * ORC_PI / 3.0, r = sqrt(3.0) / 2.0;
    out[0] = r * cos(t); out[1] = r * sin(t);
}

/* Trace one ray (pixel u, v, aperture sample a) in the vial frame at theta = 0. */
int orc_trace(const orc_geom *g, int32_t u, int32_t v, int32_t a, orc_ray *ray)
{
    memset(ray, 0, sizeof(*ray));
    double r_out = g->r_in + g->wall;
    double qx = (u - 0.5 * (g->nu - 1)) * g->pu;   /* image point Q = (qx, 0, qz) */
    double qz = (v - 0.5 * (g->nv - 1)) * g->pv;
    double stop[2];
    orc_aperture_point(g, u, v, a, stop);
    double xi = stop[0], eta = stop[1];
    double *o = ray->origin, *d = ray->d0;
    if (g->n_surf > 0) {
        double rs = 0.0;
        for (int s = 0; s < g->n_surf; ++s)
            if (g->surf[5 * s + 4] != 0.0) rs = g->surf[5 * s + 3];
        double dx = xi * rs / g->aim, dy = 1.0, dz = eta * rs / g->aim;
        double nrm = sqrt(dx * dx + dy * dy + dz * dz);
        d[0] = dx / nrm; d[1] = dy / nrm; d[2] = dz / nrm;
        o[0] = qx / g->mag; o[1] = g->obj_y; o[2] = qz / g->mag;
        if (!orc_lens_train(g, o, d)) { ray->status = 0; return 0; }
    } else if (isinf(g->pupil)) {
        /* telecentric: every ray crosses Q; the cone half-angle is atan(1/(2N)) */
        double ta = isinf(g->fnum) ? 0.0 : 1.0 / (2.0 * g->fnum);
        double dx = -xi * ta, dy = 1.0, dz = -eta * ta;
        double nrm = sqrt(dx * dx + dy * dy + dz * dz);
        d[0] = dx / nrm; d[1] = dy / nrm; d[2] = dz / nrm;
        double back = (r_out + 1.0) / d[1];
        o[0] = qx - back * d[0]; o[1] = -back * d[1]; o[2] = qz - back * d[2];
    } else {
        /* aperture stop at y = -L, diameter D = L / N, centred on the optical axis */
        double L = g->pupil;
        double D = isinf(g->fnum) ? 0.0 : L / g->fnum;
        o[0] = 0.5 * D * xi; o[1] = -L; o[2] = 0.5 * D * eta;
        double dx = qx - o[0], dy = 0.0 - o[1], dz = qz - o[2];
        double nrm = sqrt(dx * dx + dy * dy + dz * dz);
        d[0] = dx / nrm; d[1] = dy / nrm; d[2] = dz / nrm;
    }
    /* air -> glass at the outer surface */
    double tn, tf;
    if (!cylinder_roots(o, d, r_out, &tn, &tf) || tn <= 0.0) { ray->status = 0; return 0; }
    for (int i = 0; i < 3; ++i) ray->p1[i] = o[i] + tn * d[i];
    if (!refract(ray->p1, r_out, d, g->n_out, g->n_glass, ray->d1, &ray->t1)) { ray->status = -1; return -1; }
    /* glass -> resin at the inner surface */
    if (!cylinder_roots(ray->p1, ray->d1, g->r_in, &tn, &tf) || tn <= 0.0) { ray->status = 1; return 1; }
    for (int i = 0; i < 3; ++i) ray->e[i] = ray->p1[i] + tn * ray->d1[i];
    if (!refract(ray->e, g->r_in, ray->d1, g->n_glass, g->n_resin, ray->d2, &ray->t2)) { ray->status = -1; return -1; }
    /* far-side inner wall: the chord from a point on the circle along d2 */
    const double *e = ray->e, *d2 = ray->d2;
    double ell = -2.0 * (e[0] * d2[0] + e[1] * d2[1]) / (d2[0] * d2[0] + d2[1] * d2[1]);
    if (!(ell > 0.0)) { ray->status = 1; return 1; }
    ray->ell = ell;
    for (int i = 0; i < 3; ++i) ray->exit[i] = e[i] + ell * d2[i];
    double ds = g->step_vox * g->h;
    int32_t k = (int32_t)ceil(ell / ds - 1e-9);
    ray->k = k < 1 ? 1 : k;
    ray->status = 2;
    return 2;
}

/* Trilinear corners (Sec. 2.2) of a point given in index coordinates. */
typedef struct { int64_t idx[8]; double w[8]; int n; } corners8;

static void trilinear(const orc_geom *g, const double q[3], corners8 *c)
{
    double f[3]; int64_t i0[3];
    for (int ax = 0; ax < 3; ++ax) { double fl = floor(q[ax]); i0[ax] = (int64_t)fl; f[ax] = q[ax] - fl; }
    int64_t n[3] = {g->nx, g->ny, g->nz};
    c->n = 0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                int64_t ix = i0[0] + cx, iy = i0[1] + cy, iz = i0[2] + cz;
                if (ix < 0 || iy < 0 || iz < 0 || ix >= n[0] || iy >= n[1] || iz >= n[2]) continue;
                double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
                c->idx[c->n] = (iz * n[1] + iy) * n[0] + ix;
                c->w[c->n] = w;
                c->n++;
            }
}

/* Position of sample j of a traced ray after rotating the vial by theta, in index
 * coordinates, and the sample's factor w_a T1 T2 exp(-mu s_j) delta. */
static void sample(const orc_geom *g, const orc_ray *ray, int32_t j, double ct, double st,
                   double q[3], double *factor)
{
    double delta = ray->ell / ray->k;
    double s = (j + 0.5) * delta;
    double x = ray->e[0] + s * ray->d2[0];
    double y = ray->e[1] + s * ray->d2[1];
    double z = ray->e[2] + s * ray->d2[2];
    double xr = ct * x - st * y;
    double yr = st * x + ct * y;
    q[0] = xr / g->h + 0.5 * (g->nx - 1);
    q[1] = yr / g->h + 0.5 * (g->ny - 1);
    q[2] = z / g->h + 0.5 * (g->nz - 1);
    *factor = (ray->t1 * ray->t2 / g->m) * exp(-g->mu * s) * delta;
}

/* The projection exactly as Sec. 2.4 prints it: the sum, over each ray, of the voxels it
 * crosses (trilinear weights, step delta), averaged over the pixel's rays. */
static double unattenuated_factor(const orc_geom *g, const orc_ray *ray) { return (ray->ell / ray->k) / g->m; }

/* One projection pixel: y[k][v][u] = sum_a sum_j factor_j sum_corners w_c V[c]. */
double orc_adjoint_pixel(const orc_geom *g, const double *vol, int32_t k, int32_t v, int32_t u)
{
    double ct = cos(g->angles[k]), st = sin(g->angles[k]);
    double acc = 0.0;
    for (int32_t a = 0; a < g->m; ++a) {
        orc_ray ray;
        if (orc_trace(g, u, v, a, &ray) != 2) continue;
        for (int32_t j = 0; j < ray.k; ++j) {
            double q[3], fac;
            sample(g, &ray, j, ct, st, q, &fac);
            if (g->unattenuated) fac = unattenuated_factor(g, &ray);
            corners8 c;
            trilinear(g, q, &c);
            for (int i = 0; i < c.n; ++i) acc += fac * c.w[i] * vol[c.idx[i]];
        }
    }
    return acc;
}

/* Projection operator (Sec. 2.4 with Sec. 2.5's factors): volume -> projections [k][v][u]. */
void orc_adjoint(const orc_geom *g, const double *vol, double *proj)
{
    for (int32_t k = 0; k < g->n_angles; ++k)
        for (int32_t v = 0; v < g->nv; ++v)
            for (int32_t u = 0; u < g->nu; ++u)
                proj[((int64_t)k * g->nv + v) * g->nu + u] = orc_adjoint_pixel(g, vol, k, v, u);
}

/* Dose operator (Sec. 2.5): projections [k][v][u] -> dose [z][y][x], overwriting dose. */
void orc_forward(const orc_geom *g, const double *proj, double *dose)
{
    memset(dose, 0, sizeof(double) * (size_t)g->nx * g->ny * g->nz);
    for (int32_t k = 0; k < g->n_angles; ++k) {
        double ct = cos(g->angles[k]), st = sin(g->angles[k]);
        for (int32_t v = 0; v < g->nv; ++v)
            for (int32_t u = 0; u < g->nu; ++u) {
                double intensity = proj[((int64_t)k * g->nv + v) * g->nu + u];
                if (intensity == 0.0) continue;   /* adds exactly zero */
                for (int32_t a = 0; a < g->m; ++a) {
                    orc_ray ray;
                    if (orc_trace(g, u, v, a, &ray) != 2) continue;
                    for (int32_t j = 0; j < ray.k; ++j) {
                        double q[3], fac;
                        sample(g, &ray, j, ct, st, q, &fac);
                        corners8 c;
                        trilinear(g, q, &c);
                        for (int i = 0; i < c.n; ++i) dose[c.idx[i]] += intensity * fac * c.w[i];
                    }
                }
            }
    }
}

/* Dose contributions of one projection pixel (k, v, u) of intensity `intensity` (Sec. 2.5,
 * the same terms orc_forward adds for that pixel), listed instead of summed into a dense
 * volume: entry i adds val[i] to voxel idx[i].  Writes at most cap entries; returns the
 * number of contributions (more than cap means the lists were cut short). */
int64_t orc_forward_pixel(const orc_geom *g, int32_t k, int32_t v, int32_t u, double intensity, int64_t *idx,
                          double *val, int64_t cap)
{
    double ct = cos(g->angles[k]), st = sin(g->angles[k]);
    int64_t n = 0;
    for (int32_t a = 0; a < g->m; ++a) {
        orc_ray ray;
        if (orc_trace(g, u, v, a, &ray) != 2) continue;
        for (int32_t j = 0; j < ray.k; ++j) {
            double q[3], fac;
            sample(g, &ray, j, ct, st, q, &fac);
            corners8 c;
            trilinear(g, q, &c);
            for (int i = 0; i < c.n; ++i) {
                if (n < cap) { idx[n] = c.idx[i]; val[n] = intensity * fac * c.w[i]; }
                n++;
            }
        }
    }
    return n;
}

/* Samples per pass whose trilinear footprint reaches the grid (-1 < q_z < nz); the
 * rotation is about z, so the count is the same for every angle. */
uint64_t orc_sample_count(const orc_geom *g)
{
    uint64_t per_angle = 0;
    for (int32_t v = 0; v < g->nv; ++v)
        for (int32_t u = 0; u < g->nu; ++u)
            for (int32_t a = 0; a < g->m; ++a) {
                orc_ray ray;
                if (orc_trace(g, u, v, a, &ray) != 2) continue;
                double delta = ray.ell / ray.k;
                for (int32_t j = 0; j < ray.k; ++j) {
                    double s = (j + 0.5) * delta;
                    double qz = (ray.e[2] + s * ray.d2[2]) / g->h + 0.5 * (g->nz - 1);
                    if (qz > -1.0 && qz < (double)g->nz) per_angle++;
                }
            }
    return per_angle * (uint64_t)g->n_angles;
}

int32_t orc_sizeof_geom(void) { return (int32_t)sizeof(orc_geom); }
int32_t orc_sizeof_ray(void) { return (int32_t)sizeof(orc_ray); }
