// Ray generation and refraction through the vial (Sec. 2.1), once per projector, FP64.
//
// One thread per (pixel, aperture sample).  The ray leaves the aperture stop (or, for a
// telecentric projector, arrives parallel to its cone direction; or, with a lens train,
// leaves the pixel and refracts through every lens surface), meets the outer
// cylinder, refracts into the glass by the vector form of Snell's law with the
// unpolarised Fresnel transmission, does the same at the inner cylinder, and runs
// straight through the resin to the inner wall on the far side.  Everything up to the
// stored segment is FP64: the quadratic near grazing incidence and the refraction are
// where FP32 would lose the geometry.  The segment is stored in FP64, in voxel units: on a
// 768-voxel grid an FP32 entry point or direction would already misplace far samples by
// ~1e-5 voxel.
#include <math.h>

#include "internal.cuh"

namespace vamrt {
namespace {

struct d3 { double x, y, z; };

__device__ inline d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }

// Line o + t d against x^2 + y^2 = R^2.  Near and far parameters, false on a miss.
__device__ bool hit_cylinder(d3 o, d3 d, double R, double &tn, double &tf)
{
    const double a = d.x * d.x + d.y * d.y;
    const double b = 2.0 * (o.x * d.x + o.y * d.y);
    const double c = o.x * o.x + o.y * o.y - R * R;
    if (!(a > 0.0)) return false;
    const double disc = b * b - 4.0 * a * c;
    if (disc < 0.0) return false;
    // numerically stable pair of roots
    const double q = -0.5 * (b + copysign(sqrt(disc), b));
    if (q == 0.0) return false;
    const double r1 = q / a, r2 = c / q;
    tn = fmin(r1, r2);
    tf = fmax(r1, r2);
    return true;
}

// Snell's law in vector form at point p of the cylinder of radius R, index n1 -> n2.
// Returns false on total internal reflection; T = unpolarised Fresnel transmission.
__device__ bool snell(d3 p, double R, d3 d, double n1, double n2, d3 &out, double &T)
{
    d3 n = {p.x / R, p.y / R, 0.0};
    double cosi = -(n.x * d.x + n.y * d.y);
    if (cosi < 0.0) { n = -1.0 * n; cosi = -cosi; }      // normal faces the incoming ray
    const double eta = n1 / n2;
    const double k = 1.0 - eta * eta * (1.0 - cosi * cosi);
    if (k < 0.0) return false;
    const double cost = sqrt(k);
    out = eta * d + (eta * cosi - cost) * n;
    const double rs = (n1 * cosi - n2 * cost) / (n1 * cosi + n2 * cost);
    const double rp = (n1 * cost - n2 * cosi) / (n1 * cost + n2 * cosi);
    T = 1.0 - 0.5 * (rs * rs + rp * rp);
    return true;
}

__device__ inline double dot3(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Lens train (Sec. 2.1: rays refract at every optical element on the way to the vial).
// Surface k: sv[5k..5k+4] = vertex y, radius of curvature (centre at y + radius; INF =
// plane), index behind, clear semi-aperture, stop flag.  The ray (o, d) starts in front
// of the first surface in the outside medium; on success o is its point on the last
// surface and d its direction behind it.  False when a surface is missed, a clear
// aperture blocks the ray, or it is totally reflected.
__device__ bool through_lenses(const double *sv, int n_surf, double n0, d3 &o, d3 &d)
{
    double n_in = n0;
    for (int k = 0; k < n_surf; ++k) {
        const double yv = sv[5 * k], R = sv[5 * k + 1], n_out = sv[5 * k + 2], ap = sv[5 * k + 3];
        const bool iris = sv[5 * k + 4] != 0.0;
        double t = -1.0;
        d3 c = {0.0, yv + R, 0.0};
        if (isinf(R)) {
            if (d.y != 0.0) t = (yv - o.y) / d.y;
        } else {
            // |o + t d - c| = |R|: of the two crossings take the one on the vertex's side of c
            const d3 oc = {o.x - c.x, o.y - c.y, o.z - c.z};
            const double half_b = dot3(d, oc);
            const double disc = half_b * half_b - (dot3(oc, oc) - R * R);
            if (disc >= 0.0) {
                const double root = sqrt(disc);
                const double ta = -half_b - root, tb = -half_b + root;
                if (ta > 0.0 && (o.y + ta * d.y - c.y) * (yv - c.y) > 0.0) t = ta;
                else if (tb > 0.0 && (o.y + tb * d.y - c.y) * (yv - c.y) > 0.0) t = tb;
            }
        }
        if (!(t > 0.0)) return false;
        const d3 p = o + t * d;
        if (p.x * p.x + p.z * p.z > ap * ap) return false;           // vignetted
        if (!iris) {
            d3 nrm = isinf(R) ? d3{0.0, 1.0, 0.0} : d3{p.x / R, (p.y - c.y) / R, p.z / R};
            double cosi = -dot3(nrm, d);
            if (cosi < 0.0) { nrm = -1.0 * nrm; cosi = -cosi; }
            const double mu = n_in / n_out;
            const double rad = 1.0 - mu * mu * (1.0 - cosi * cosi);
            if (rad < 0.0) return false;
            d = mu * d + (mu * cosi - sqrt(rad)) * nrm;
        }
        o = p;
        n_in = n_out;
    }
    return true;
}

// ---------------------------------------------------------------------------------
// aperture-stop samples (Sec. 2.1: a pixel's rays leave points of the stop)
// ---------------------------------------------------------------------------------

// splitmix64 as published (Steele, Lea and Flood; Vigna's form): Weyl step, then mix.
__device__ __forceinline__ unsigned long long mix64(unsigned long long state)
{
    unsigned long long z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// uniform in [0, 1): 53 high bits of the hash of (pixel, ray, component)
__device__ double jitter01(unsigned long long seed, int u, int v, int a, int c)
{
    const unsigned long long key = (unsigned long long)(unsigned)u | ((unsigned long long)(unsigned)v << 20) |
                                   ((unsigned long long)(unsigned)a << 40) | ((unsigned long long)(unsigned)c << 56);
    return (double)(mix64(seed ^ key) >> 11) * 0x1.0p-53;
}

// Shirley-Chiu concentric square-to-disk map of (s, t) in [-1,1]^2
__device__ void square_to_disk(double s, double t, double &x, double &y)
{
    const double quarter = 0.78539816339744830962;   // pi / 4
    double rad = 0.0, ang = 0.0;
    if (s != 0.0 || t != 0.0) {
        if (fabs(s) > fabs(t)) {
            rad = s;
            ang = quarter * (t / s);
        } else {
            rad = t;
            ang = 2.0 * quarter - quarter * (s / t);
        }
    }
    double sn, cs;
    sincos(ang, &sn, &cs);
    x = rad * cs;
    y = rad * sn;
}

__device__ void stop_point(const TraceParams &P, int u, int v, int a, double &xi, double &et)
{
    const int ju = P.per_pixel ? u : 0, jv = P.per_pixel ? v : 0;
    xi = 0.0;
    et = 0.0;
    switch (P.aperture) {
    case VAMRT_APERTURE_LIST:
        xi = P.pupil_xy[2 * a];
        et = P.pupil_xy[2 * a + 1];
        break;
    case VAMRT_APERTURE_STRATIFIED: {
        const int n = P.strat_n, i = a / n, k = a - (a / n) * n;
        const double s = 2.0 * ((double)i + jitter01(P.seed, ju, jv, a, 0)) / n - 1.0;
        const double t = 2.0 * ((double)k + jitter01(P.seed, ju, jv, a, 1)) / n - 1.0;
        square_to_disk(s, t, xi, et);
        break;
    }
    case VAMRT_APERTURE_SUNFLOWER: {
        const double pi = 3.14159265358979323846;
        const double golden = pi * (3.0 - sqrt(5.0));
        const double r = sqrt(((double)a + 0.5) / P.M);
        const double ang = (double)a * golden + 2.0 * pi * jitter01(P.seed, ju, jv, 0, 0);
        xi = r * cos(ang);
        et = r * sin(ang);
        break;
    }
    case VAMRT_APERTURE_HEX: {
        // hexagonal lattice of spacing 1/2 inside the unit disk: centre, inner ring of 6 at
        // 1/2, outer ring of 6 at sqrt(3)/2 turned by 30 degrees
        const double pi = 3.14159265358979323846;
        if (a >= 1 && a <= 6) {
            xi = 0.5 * cos((a - 1) * (pi / 3.0));
            et = 0.5 * sin((a - 1) * (pi / 3.0));
        } else if (a >= 7) {
            const double ang = pi / 6.0 + (a - 7) * (pi / 3.0);
            xi = 0.5 * sqrt(3.0) * cos(ang);
            et = 0.5 * sqrt(3.0) * sin(ang);
        }
        break;
    }
    default:   // VAMRT_APERTURE_CHIEF
        break;
    }
}

__global__ void raytable_kernel(TraceParams P, double4_32a *__restrict__ A, double4_32a *__restrict__ B,
                                int2 *__restrict__ J, unsigned long long *__restrict__ counters)
{
    const int64_t n_rays = (int64_t)P.nu * P.nv * P.M;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int u = (int)(r % P.nu);
    const int v = (int)((r / P.nu) % P.nv);
    const int a = (int)(r / ((int64_t)P.nu * P.nv));

    A[r] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    B[r] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    J[r] = make_int2(0, 0);

    // image point of the pixel in the best-focus plane y = 0
    const d3 Q = {(u - 0.5 * (P.nu - 1)) * P.pu, 0.0, (v - 0.5 * (P.nv - 1)) * P.pv};
    double xi, et;
    stop_point(P, u, v, a, xi, et);
    d3 o, d;
    if (P.n_surf > 0) {
        // pixel in the object plane, launched telecentric in object space towards the stop
        o = {Q.x / P.mag, P.obj_y, Q.z / P.mag};
        d = {xi * P.stop_r / P.aim, 1.0, et * P.stop_r / P.aim};
        d = (1.0 / sqrt(dot3(d, d))) * d;
        if (!through_lenses(P.surf, P.n_surf, P.n_out, o, d)) return;          // blocked
    } else if (P.telecentric) {
        const double t = P.chief_only ? 0.0 : 1.0 / (2.0 * P.f_number);
        d = {-xi * t, 1.0, -et * t};
        d = (1.0 / sqrt(d.x * d.x + d.y * d.y + d.z * d.z)) * d;
        const double back = (P.r_out + 1.0) / d.y;        // start in front of the vial
        o = Q + (-back) * d;
    } else {
        const double D = P.chief_only ? 0.0 : P.pupil_mm / P.f_number;
        o = {0.5 * D * xi, -P.pupil_mm, 0.5 * D * et};
        d = {Q.x - o.x, Q.y - o.y, Q.z - o.z};
        d = (1.0 / sqrt(d.x * d.x + d.y * d.y + d.z * d.z)) * d;
    }
    double tn, tf, T1, T2;
    if (!hit_cylinder(o, d, P.r_out, tn, tf) || !(tn > 0.0)) return;         // misses the vial
    const d3 p1 = o + tn * d;
    d3 dg;
    if (!snell(p1, P.r_out, d, P.n_out, P.n_glass, dg, T1)) return;
    if (!hit_cylinder(p1, dg, P.r_in, tn, tf) || !(tn > 0.0)) return;       // wall only
    const d3 e = p1 + tn * dg;
    d3 dr;
    if (!snell(e, P.r_in, dg, P.n_glass, P.n_resin, dr, T2)) return;        // TIR: dropped
    // far side: chord of the circle from e along dr
    const double ell = -2.0 * (e.x * dr.x + e.y * dr.y) / (dr.x * dr.x + dr.y * dr.y);
    if (!(ell > 0.0)) return;
    int K = (int)ceil(ell / P.ds - 1e-9);
    if (K < 1) K = 1;
    const double delta = ell / K;

    // samples whose trilinear footprint reaches the grid in z: -1 < q_z < nz.  q_z is
    // linear in j, so they form one run.  The expression is evaluated without fused
    // multiply-adds so that it rounds like a plain FP64 evaluation.
    const double zc = 0.5 * (P.nz - 1);
    int jlo = K, jhi = 0;
    for (int j = 0; j < K; ++j) {
        const double s = __dmul_rn((double)j + 0.5, delta);
        const double qz = __dadd_rn(__ddiv_rn(__dadd_rn(e.z, __dmul_rn(s, dr.z)), P.h), zc);
        if (qz > -1.0 && qz < (double)P.nz) {
            if (j < jlo) jlo = j;
            jhi = j + 1;
        }
    }
    if (jhi <= jlo) { jlo = 0; jhi = 0; }

    const double inv_h = 1.0 / P.h;
    A[r] = make_double4_32a(e.x * inv_h, e.y * inv_h, e.z * inv_h, delta * inv_h);
    B[r] = make_double4_32a(dr.x, dr.y, dr.z, T1 * T2 * delta / P.M);
    J[r] = make_int2(jlo, jhi);
    atomicAdd(&counters[0], 1ull);
    atomicAdd(&counters[1], (unsigned long long)(jhi - jlo));
}

}  // namespace

cudaError_t launch_raytable(const TraceParams &T, double4_32a *A, double4_32a *B, int2 *J,
                            unsigned long long *counters, cudaStream_t s)
{
    const int64_t n = (int64_t)T.nu * T.nv * T.M;
    const int threads = 128;
    const int64_t blocks = (n + threads - 1) / threads;
    raytable_kernel<<<(unsigned)blocks, threads, 0, s>>>(T, A, B, J, counters);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
