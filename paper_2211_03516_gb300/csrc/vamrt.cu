// C-ABI entry points: argument validation, the projector handle, dispatch, and the
// optimiser's host loop.  No exception or exit() crosses this boundary.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "internal.cuh"

namespace {

thread_local char g_err[512] = "";
std::atomic<uint64_t> g_launches{0};

vamrt_status fail(vamrt_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

vamrt_status cuda_fail(cudaError_t e, const char *where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(VAMRT_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(VAMRT_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call, where)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);  \
    } while (0)

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

vamrt_status validate(const vamrt_geometry *g)
{
    if (!g) return fail(VAMRT_EINVAL, "geometry is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail(VAMRT_EINVAL, "grid extents must be >= 1");
    if (g->nu < 1 || g->nv < 1) return fail(VAMRT_EINVAL, "pixel array extents must be >= 1");
    if (g->n_angles < 1 || g->n_angles > 65535) return fail(VAMRT_EINVAL, "n_angles must be in 1..65535");
    if (g->nv > 4 * 65535) return fail(VAMRT_EINVAL, "nv too large");
    if (!finite_pos(g->voxel_mm)) return fail(VAMRT_EINVAL, "voxel_mm must be finite and > 0");
    if (!finite_pos(g->pixel_u_mm) || !finite_pos(g->pixel_v_mm))
        return fail(VAMRT_EINVAL, "pixel pitches must be finite and > 0");
    if (!(g->pupil_mm > 0.0) || isnan(g->pupil_mm)) return fail(VAMRT_EINVAL, "pupil_mm must be > 0 or INFINITY");
    if (!(g->f_number > 0.0) || isnan(g->f_number)) return fail(VAMRT_EINVAL, "f_number must be > 0 or INFINITY");
    if (g->rays_per_pixel < 1 || g->rays_per_pixel > 4096) return fail(VAMRT_EINVAL, "rays_per_pixel must be 1..4096");
    if (g->aperture_flags & ~VAMRT_JITTER_PER_PIXEL) return fail(VAMRT_EINVAL, "unknown aperture_flags");
    switch (g->aperture) {
    case VAMRT_APERTURE_LIST:
        if (!g->pupil_xy && g->rays_per_pixel != 1)
            return fail(VAMRT_EINVAL, "pupil_xy may be NULL only with one ray per pixel");
        break;
    case VAMRT_APERTURE_CHIEF:
        if (g->rays_per_pixel != 1) return fail(VAMRT_EINVAL, "the chief-ray aperture has one ray per pixel");
        break;
    case VAMRT_APERTURE_STRATIFIED: {
        const int n = (int)lround(sqrt((double)g->rays_per_pixel));
        if (n * n != g->rays_per_pixel) return fail(VAMRT_EINVAL, "stratified aperture needs n^2 rays per pixel");
        break;
    }
    case VAMRT_APERTURE_SUNFLOWER:
        break;
    case VAMRT_APERTURE_HEX:
        if (g->rays_per_pixel != 13) return fail(VAMRT_EINVAL, "the hexagonal aperture has 13 rays per pixel");
        break;
    default:
        return fail(VAMRT_EINVAL, "unknown aperture pattern %d", g->aperture);
    }
    if (g->nu >= (1 << 20) || g->nv >= (1 << 20)) return fail(VAMRT_EINVAL, "nu and nv must be below 2^20");
    if (g->aperture == VAMRT_APERTURE_LIST && g->pupil_xy)
        for (int a = 0; a < g->rays_per_pixel; ++a) {
            const double x = g->pupil_xy[2 * a], y = g->pupil_xy[2 * a + 1];
            if (!isfinite(x) || !isfinite(y) || x * x + y * y > 1.0 + 1e-12)
                return fail(VAMRT_EINVAL, "pupil sample %d is not in the unit disk", a);
        }
    if (!finite_pos(g->r_inner_mm)) return fail(VAMRT_EINVAL, "r_inner_mm must be finite and > 0");
    if (!isfinite(g->wall_mm) || g->wall_mm < 0.0) return fail(VAMRT_EINVAL, "wall_mm must be finite and >= 0");
    if (!finite_pos(g->n_outside) || !finite_pos(g->n_glass) || !finite_pos(g->n_resin))
        return fail(VAMRT_EINVAL, "refractive indices must be finite and > 0");
    if (!isfinite(g->mu_per_mm) || g->mu_per_mm < 0.0) return fail(VAMRT_EINVAL, "mu_per_mm must be finite and >= 0");
    if (g->step_vox != 0.0 && (!finite_pos(g->step_vox) || g->step_vox > 8.0))
        return fail(VAMRT_EINVAL, "step_vox must be in (0, 8] (0 = default 0.5)");
    if (g->angles_rad)
        for (int k = 0; k < g->n_angles; ++k)
            if (!isfinite(g->angles_rad[k])) return fail(VAMRT_EINVAL, "angle %d is not finite", k);
    if (g->n_surfaces < 0 || g->n_surfaces > 64) return fail(VAMRT_EINVAL, "n_surfaces must be in 0..64");
    if (g->n_surfaces > 0) {
        if (!g->surfaces) return fail(VAMRT_EINVAL, "surfaces is NULL");
        if (!isfinite(g->object_y_mm) || !(g->object_y_mm < g->surfaces[0].y_mm))
            return fail(VAMRT_EINVAL, "object_y_mm must be finite and before the first surface");
        if (!isfinite(g->magnification) || g->magnification == 0.0)
            return fail(VAMRT_EINVAL, "magnification must be finite and nonzero");
        if (!finite_pos(g->aim_mm)) return fail(VAMRT_EINVAL, "aim_mm must be finite and > 0");
        int stops = 0;
        for (int s = 0; s < g->n_surfaces; ++s) {
            const vamrt_surface &S = g->surfaces[s];
            if (!isfinite(S.y_mm) || (s > 0 && !(S.y_mm > g->surfaces[s - 1].y_mm)))
                return fail(VAMRT_EINVAL, "surface %d: y_mm must be finite and increasing", s);
            if (isnan(S.radius_mm) || S.radius_mm == 0.0 || (isinf(S.radius_mm) && S.radius_mm < 0.0))
                return fail(VAMRT_EINVAL, "surface %d: radius_mm must be nonzero (INFINITY = plane)", s);
            if (!finite_pos(S.n_after) || !finite_pos(S.clear_mm))
                return fail(VAMRT_EINVAL, "surface %d: n_after and clear_mm must be finite and > 0", s);
            if (S.is_stop) {
                ++stops;
                if (!isinf(S.radius_mm)) return fail(VAMRT_EINVAL, "surface %d: the stop must be a plane", s);
            }
        }
        if (stops != 1) return fail(VAMRT_EINVAL, "the lens train needs exactly one stop (found %d)", stops);
        if (g->surfaces[g->n_surfaces - 1].n_after != g->n_outside)
            return fail(VAMRT_EINVAL, "the last surface must leave the ray in the outside medium (n_outside)");
        if (!(g->surfaces[g->n_surfaces - 1].y_mm < -(g->r_inner_mm + g->wall_mm)))
            return fail(VAMRT_EINVAL, "the lens train must end before the vial");
    }
    const int nmin = g->nx < g->ny ? g->nx : g->ny;
    if (!(g->r_inner_mm / g->voxel_mm <= 0.5 * (nmin + 1) - 0.01))
        return fail(VAMRT_EINVAL, "grid (%d x %d voxels of %g mm) does not enclose the resin radius %g mm",
                    g->nx, g->ny, g->voxel_mm, g->r_inner_mm);
    const int64_t pad = (int64_t)(((g->nx + 2 + 3) / 4) * 4) * (g->ny + 2) * (g->nz + 2);
    if (pad >= (int64_t)1 << 31) return fail(VAMRT_EINVAL, "grid too large (padded voxels must fit int32)");
    const int64_t rays = (int64_t)g->nu * g->nv * g->rays_per_pixel;
    if (rays >= (int64_t)1 << 31) return fail(VAMRT_EINVAL, "too many rays");
    // rays of up to ~2 R / step samples; keep j and (j + 1/2) exact in FP32
    const double step = g->step_vox == 0.0 ? 0.5 : g->step_vox;
    if (2.0 * g->r_inner_mm / (step * g->voxel_mm) > 4.0e6) return fail(VAMRT_EINVAL, "too many samples per ray");
    return VAMRT_OK;
}

vamrt_status check_dtype(vamrt_dtype d)
{
    if (d != VAMRT_F32 && d != VAMRT_BF16 && d != VAMRT_F16) return fail(VAMRT_EINVAL, "unknown dtype %d", (int)d);
    return VAMRT_OK;
}

void release(vamrt_projector *p)
{
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->tabA);
    cudaFree(p->tabB);
    cudaFree(p->tabJ);
    cudaFree(p->cs);
    cudaFree(p->scratch);
    cudaFree(p->red);
    cudaFree(p->hist);
    cudaFree(p->dmax);
    if (p->host_err) cudaFreeHost(p->host_err);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

struct Guard {
    vamrt_projector *p;
    ~Guard() { release(p); }
};

}  // namespace

namespace vamrt {
void count_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace vamrt

extern "C" {

uint64_t vamrt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *vamrt_status_string(vamrt_status s)
{
    switch (s) {
    case VAMRT_OK: return "ok";
    case VAMRT_EINVAL: return "invalid argument";
    case VAMRT_EUNSUPPORTED: return "unsupported";
    case VAMRT_ECUDA: return "CUDA error";
    case VAMRT_ENOMEM: return "out of device memory";
    case VAMRT_NOT_CONVERGED: return "not converged";
    case VAMRT_NUMERIC: return "numeric error (NaN/Inf or zero dose)";
    }
    return "unknown status";
}

const char *vamrt_last_error(void) { return g_err; }

vamrt_status vamrt_make_projector(const vamrt_geometry *geom, void *stream, vamrt_projector **out)
{
    g_err[0] = 0;
    if (!out) return fail(VAMRT_EINVAL, "out is NULL");
    *out = nullptr;
    vamrt_status st = validate(geom);
    if (st != VAMRT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    vamrt_projector *p = new (std::nothrow) vamrt_projector();
    if (!p) return fail(VAMRT_ENOMEM, "host allocation failed");
    Guard guard{p};
    p->g = *geom;
    p->g.pupil_xy = nullptr;          // host arrays, used only while tracing below
    p->g.angles_rad = nullptr;
    p->g.surfaces = nullptr;          // host array, used only while tracing below
    if (p->g.step_vox == 0.0) p->g.step_vox = 0.5;
    const vamrt_geometry &g = p->g;
    const int M = g.rays_per_pixel;

    CK(cudaGetDevice(&p->device), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device), "cudaDeviceGetAttribute");
    {
        // load the allocation-free dose entry point's static accumulator here, where
        // allocating is expected, so that vamrt_forward_dose_static never allocates
        float *static_acc = nullptr;
        CK(vamrt::static_acc_address(p->device, &static_acc), "static accumulator");
    }
    p->n_rays = (int64_t)g.nu * g.nv * M;
    const int px = ((g.nx + 2 + 3) / 4) * 4;   // rows padded to 16-byte groups
    p->pad_elems = (int64_t)px * (g.ny + 2) * (g.nz + 2);

    CK(cudaMalloc(&p->tabA, sizeof(double4_32a) * p->n_rays), "cudaMalloc(ray table)");
    CK(cudaMalloc(&p->tabB, sizeof(double4_32a) * p->n_rays), "cudaMalloc(ray table)");
    CK(cudaMalloc(&p->tabJ, sizeof(int2) * p->n_rays), "cudaMalloc(ray table)");
    CK(cudaMalloc(&p->cs, sizeof(double2) * g.n_angles), "cudaMalloc(angles)");
    CK(cudaMalloc(&p->scratch, sizeof(float) * p->pad_elems), "cudaMalloc(scratch volume)");
    CK(cudaMalloc(&p->red, sizeof(double) * (vamrt::kRedBlocks + 8)), "cudaMalloc(reduction)");
    CK(cudaMalloc(&p->hist, sizeof(double) * vamrt::kMaxHistory), "cudaMalloc(history)");
    CK(cudaMalloc(&p->dmax, sizeof(float) * 4), "cudaMalloc(dmax)");
    CK(cudaMallocHost(&p->host_err, 4 * sizeof(double)), "cudaMallocHost");   // E and the 3 VER counts
    p->device_bytes = (sizeof(double4_32a) * 2 + sizeof(int2)) * (uint64_t)p->n_rays + sizeof(double2) * g.n_angles +
                      sizeof(float) * (uint64_t)p->pad_elems;

    // angle table, FP64 on the host then rounded
    double2 *hcs = (double2 *)malloc(sizeof(double2) * g.n_angles);
    if (!hcs) return fail(VAMRT_ENOMEM, "host allocation failed");
    for (int k = 0; k < g.n_angles; ++k) {
        const double th = geom->angles_rad ? geom->angles_rad[k] : 2.0 * M_PI * k / g.n_angles;
        hcs[k] = make_double2(cos(th), sin(th));
    }
    cudaError_t e = cudaMemcpyAsync(p->cs, hcs, sizeof(double2) * g.n_angles, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(hcs);
    if (e != cudaSuccess) return cuda_fail(e, "angle table upload");

    // pupil samples, counters and the lens train (5 doubles per surface) in one temporary
    // device block
    const size_t pupil_bytes = sizeof(double) * 2 * M;
    const int n_surf = geom->n_surfaces;
    std::vector<double> hsurf(5 * (size_t)n_surf);
    double stop_r = 0.0;
    for (int k = 0; k < n_surf; ++k) {
        const vamrt_surface &S = geom->surfaces[k];
        hsurf[5 * k] = S.y_mm; hsurf[5 * k + 1] = S.radius_mm; hsurf[5 * k + 2] = S.n_after;
        hsurf[5 * k + 3] = S.clear_mm; hsurf[5 * k + 4] = S.is_stop ? 1.0 : 0.0;
        if (S.is_stop) stop_r = S.clear_mm;
    }
    const size_t surf_bytes = sizeof(double) * hsurf.size();
    void *tmp = nullptr;
    CK(cudaMalloc(&tmp, pupil_bytes + surf_bytes + 2 * sizeof(unsigned long long)), "cudaMalloc(tmp)");
    double *d_pupil = (double *)tmp;
    double *d_surf = d_pupil + 2 * M;
    unsigned long long *d_cnt = (unsigned long long *)((char *)tmp + pupil_bytes + surf_bytes);
    const bool listed = geom->aperture == VAMRT_APERTURE_LIST && geom->pupil_xy;
    e = listed ? cudaMemcpyAsync(d_pupil, geom->pupil_xy, pupil_bytes, cudaMemcpyHostToDevice, s)
               : cudaMemsetAsync(d_pupil, 0, pupil_bytes, s);
    if (e == cudaSuccess && n_surf > 0)
        e = cudaMemcpyAsync(d_surf, hsurf.data(), surf_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 2 * sizeof(unsigned long long), s);

    vamrt::TraceParams T;
    T.pupil_xy = d_pupil;
    T.aperture = geom->aperture;
    T.per_pixel = (geom->aperture_flags & VAMRT_JITTER_PER_PIXEL) ? 1 : 0;
    T.seed = geom->seed;
    T.strat_n = (int)lround(sqrt((double)M));
    T.nu = g.nu; T.nv = g.nv; T.M = M; T.nz = g.nz;
    T.pu = g.pixel_u_mm; T.pv = g.pixel_v_mm;
    T.pupil_mm = g.pupil_mm; T.f_number = g.f_number;
    T.telecentric = isinf(g.pupil_mm) ? 1 : 0;
    T.chief_only = isinf(g.f_number) ? 1 : 0;
    T.r_in = g.r_inner_mm; T.r_out = g.r_inner_mm + g.wall_mm;
    T.n_out = g.n_outside; T.n_glass = g.n_glass; T.n_resin = g.n_resin;
    T.h = g.voxel_mm; T.ds = g.step_vox * g.voxel_mm;
    T.surf = d_surf; T.n_surf = n_surf;
    T.obj_y = geom->object_y_mm; T.mag = geom->magnification; T.aim = geom->aim_mm; T.stop_r = stop_r;
    if (e == cudaSuccess) e = vamrt::launch_raytable(T, p->tabA, p->tabB, p->tabJ, d_cnt, s);
    unsigned long long cnt[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "ray table build");
    p->rays_in_resin = (int64_t)cnt[0];
    p->samples_per_angle = cnt[1];

    vamrt::OpParams &P = p->op;
    P.A = p->tabA; P.B = p->tabB; P.J = p->tabJ; P.cs = p->cs;
    P.nu = g.nu; P.nv = g.nv; P.M = M; P.n_angles = g.n_angles;
    P.nx = g.nx; P.ny = g.ny; P.nz = g.nz;
    P.px = px; P.py = g.ny + 2; P.pz = g.nz + 2;
    P.cx = 0.5 * (g.nx - 1) + 1.0;
    P.cy = 0.5 * (g.ny - 1) + 1.0;
    P.cz = 0.5 * (g.nz - 1) + 1.0;
    P.neg_mu_vox_log2e = (float)(-g.mu_per_mm * g.voxel_mm * M_LOG2E);
    P.h_over_m = (float)(g.voxel_mm / M);
    // chunk 0 starts one voxel in front of the resin cylinder
    P.y0 = (float)(-g.r_inner_mm / g.voxel_mm - 1.0);
    // a segment crosses the (-1,1)^3 neighbourhood of a voxel over at most 2 sqrt(3)
    // voxels; consecutive samples are more than step_vox / 2 apart (K = ceil(ell/ds))
    P.cell_bound = (float)fmax(2.0, floor(4.0 * sqrt(3.0) / g.step_vox) + 1.0);

    guard.p = nullptr;
    *out = p;
    return VAMRT_OK;
}

void vamrt_destroy_projector(vamrt_projector *p) { release(p); }

vamrt_status vamrt_get_info(const vamrt_projector *p, vamrt_info *info)
{
    if (!p || !info) return fail(VAMRT_EINVAL, "NULL argument");
    info->n_rays = p->n_rays;
    info->rays_in_resin = p->rays_in_resin;
    info->samples_per_pass = p->samples_per_angle * (uint64_t)p->g.n_angles;
    info->scratch_bytes = p->device_bytes;
    return VAMRT_OK;
}

vamrt_status vamrt_sample_count(const vamrt_projector *p, uint64_t *n)
{
    if (!p || !n) return fail(VAMRT_EINVAL, "NULL argument");
    *n = p->samples_per_angle * (uint64_t)p->g.n_angles;
    return VAMRT_OK;
}

vamrt_status vamrt_adjoint(vamrt_projector *p, const void *vol, vamrt_dtype vol_dtype, void *proj,
                           vamrt_dtype proj_dtype, uint32_t flags, void *stream)
{
    if (!p || !vol || !proj) return fail(VAMRT_EINVAL, "NULL argument");
    if (check_dtype(vol_dtype) || check_dtype(proj_dtype)) return VAMRT_EINVAL;
    if (flags & ~(VAMRT_ACCUMULATE | VAMRT_CLAMP_NONNEG | VAMRT_UNATTENUATED))
        return fail(VAMRT_EINVAL, "unknown flags 0x%x", flags);
    cudaStream_t s = (cudaStream_t)stream;
    CK(vamrt::launch_pad(p, vol, vol_dtype, s), "pad kernel");
    CK(vamrt::launch_adjoint(p, vol_dtype, proj, proj_dtype, flags, s), "adjoint kernel");
    return VAMRT_OK;
}

vamrt_status vamrt_forward_dose(vamrt_projector *p, const void *proj, vamrt_dtype proj_dtype, void *dose,
                                vamrt_dtype dose_dtype, uint32_t flags, void *stream)
{
    if (!p || !proj || !dose) return fail(VAMRT_EINVAL, "NULL argument");
    if (check_dtype(proj_dtype) || check_dtype(dose_dtype)) return VAMRT_EINVAL;
    if (flags & ~VAMRT_ACCUMULATE) return fail(VAMRT_EINVAL, "unknown flags 0x%x", flags);
    cudaStream_t s = (cudaStream_t)stream;
    CK(vamrt::launch_forward(p, proj, proj_dtype, s), "forward kernel");
    CK(vamrt::launch_unpad(p, dose, dose_dtype, flags, s), "unpad kernel");
    return VAMRT_OK;
}

namespace {

// VAMRT_OPT_GRADIENT: projected Adam steps on the thresholded dose loss, the gradient
// A^T dL/dD from the projection operator (the differentiable path), from the caller's
// starting projections.  Validation common to all modes is done by the caller.
vamrt_status optimize_gradient(vamrt_projector *p, const float *target, float *model, void *proj, void *dose,
                               const vamrt_opt_params *params, vamrt_opt_report *report, cudaStream_t s)
{
    const vamrt_dtype pdt = params->proj_dtype, ddt = params->dose_dtype;
    if (pdt == VAMRT_F16) return fail(VAMRT_EUNSUPPORTED, "gradient mode stores projections as F32 or BF16");
    if (params->momentum != 0.0) return fail(VAMRT_EINVAL, "momentum is not used in gradient mode");
    const bool dflt = params->d_l == 0.0 && params->d_h == 0.0;
    const double d_l = dflt ? 0.8 : params->d_l, d_h = dflt ? 1.0 : params->d_h;
    if (!(d_l >= 0.0 && d_h > d_l)) return fail(VAMRT_EINVAL, "thresholds must satisfy 0 <= d_l < d_h");
    const double step = params->step == 0.0 ? 0.8 : params->step;
    if (!(step > 0.0 && step <= 16.0)) return fail(VAMRT_EINVAL, "gradient-mode step must be in (0, 16] (0 = 0.8)");
    const vamrt_geometry &g = p->g;
    const int64_t n = (int64_t)g.n_angles * g.nv * g.nu;
    const int64_t nvox = (int64_t)g.nx * g.ny * g.nz;

    // FP32 state for this call: Adam moments, the projection gradient and (BF16 storage)
    // the master projections
    float *state = nullptr;
    const int64_t n_state = (pdt == VAMRT_F32 ? 3 : 4) * n;
    if (cudaMalloc(&state, sizeof(float) * n_state) != cudaSuccess) {
        cudaGetLastError();
        return fail(VAMRT_ENOMEM, "gradient mode: %lld bytes of optimiser state", (long long)(sizeof(float) * n_state));
    }
    struct Free {
        float *q;
        ~Free() { cudaFree(q); }
    } free_state{state};
    float *mom1 = state, *mom2 = state + n, *gradp = state + 2 * n;
    float *master = pdt == VAMRT_F32 ? (float *)proj : state + 3 * n;
    CK(cudaMemsetAsync(mom1, 0, sizeof(float) * 2 * n, s), "cudaMemsetAsync");

    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() { for (int i = 0; i < 5; ++i) if (e[i]) cudaEventDestroy(e[i]); }
    } evguard{ev};
    if (params->timing)
        for (int i = 0; i < 5; ++i) CK(cudaEventCreate(&ev[i]), "cudaEventCreate");
    double *sc2 = p->red + vamrt::kRedBlocks + 1;     // {count, sum}
    double *loss3 = p->red + vamrt::kRedBlocks + 1;   // {L, 1/|P|, 1/|Q|}
    long long *ver3 = reinterpret_cast<long long *>(p->red + vamrt::kRedBlocks + 5);
    struct Checked {
        double err;
        long long ver3[3];
    };
    Checked *host = reinterpret_cast<Checked *>(p->host_err);
    double t_adj = 0.0, t_fwd = 0.0, t_upd = 0.0;
    if (params->timing) CK(cudaEventRecord(ev[0], s), "cudaEventRecord");

    // scale the start so that the part's mean dose is 1 (the thresholds' scale)
    CK(vamrt::launch_forward(p, proj, pdt, s), "forward kernel");
    CK(vamrt::launch_unpad(p, dose, ddt, 0u, s), "unpad kernel");
    CK(vamrt::launch_masked_sum(p, dose, ddt, target, nvox, sc2, s), "masked sum");
    double cnt[2];
    CK(cudaMemcpyAsync(cnt, sc2, sizeof(cnt), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (!(cnt[0] > 0.0)) return fail(VAMRT_EINVAL, "gradient mode: the target has no part voxels");
    if (!(cnt[1] > 0.0) || !isfinite(cnt[1]))
        return fail(VAMRT_NUMERIC, "gradient mode: the starting projections give the part no dose");
    CK(vamrt::launch_scale_master(p, proj, pdt, master, n, (float)(cnt[0] / cnt[1]), s), "scale kernel");
    // Adam step: `step` times the mean positive projection
    CK(vamrt::launch_masked_sum(p, master, VAMRT_F32, nullptr, n, sc2, s), "masked sum");
    CK(cudaMemcpyAsync(cnt, sc2, sizeof(cnt), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (!(cnt[0] > 0.0)) return fail(VAMRT_NUMERIC, "gradient mode: no positive starting projection");
    const float lr = (float)(step * cnt[1] / cnt[0]);
    if (params->timing) {
        CK(cudaEventRecord(ev[1], s), "cudaEventRecord");
        CK(cudaEventSynchronize(ev[1]), "cudaEventSynchronize");
        float ms;
        CK(cudaEventElapsedTime(&ms, ev[0], ev[1]), "cudaEventElapsedTime");
        t_fwd += ms;
    }

    int it = 0;
    double err = NAN, ver = NAN;
    bool converged = false;
    std::vector<double> vers((size_t)params->max_iter, NAN);
    for (; it < params->max_iter;) {
        if (params->timing) CK(cudaEventRecord(ev[0], s), "cudaEventRecord");
        // D = A g (stored in dose_dtype); L and dL/dD (FP32, in the model buffer)
        CK(vamrt::launch_forward(p, proj, pdt, s), "forward kernel");
        CK(vamrt::launch_unpad(p, dose, ddt, 0u, s), "unpad kernel");
        if (params->timing) CK(cudaEventRecord(ev[1], s), "cudaEventRecord");
        CK(vamrt::launch_threshold_loss(p, dose, ddt, target, (float)d_l, (float)d_h, loss3, model, VAMRT_F32, s),
           "threshold loss");
        CK(cudaMemcpyAsync(p->hist + it, loss3, sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        if (params->timing) CK(cudaEventRecord(ev[2], s), "cudaEventRecord");
        // the projections' gradient A^T dL/dD
        CK(vamrt::launch_pad(p, model, VAMRT_F32, s), "pad kernel");
        CK(vamrt::launch_adjoint(p, VAMRT_F32, gradp, VAMRT_F32, 0u, s), "adjoint kernel");
        if (params->timing) CK(cudaEventRecord(ev[3], s), "cudaEventRecord");
        // projected Adam step on the FP32 master (g >= 0), storage copy refreshed
        CK(vamrt::nn_adam(master, gradp, mom1, mom2, pdt == VAMRT_BF16 ? proj : nullptr, n, lr, 0.9f, 0.999f, 1e-12f,
                          it + 1, true, s),
           "adam kernel");
        if (params->timing) {
            CK(cudaEventRecord(ev[4], s), "cudaEventRecord");
            CK(cudaEventSynchronize(ev[4]), "cudaEventSynchronize");
            float ms[4];
            for (int i = 0; i < 4; ++i) CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]), "cudaEventElapsedTime");
            t_fwd += ms[0];
            t_upd += ms[1] + ms[3];
            t_adj += ms[2];
        }
        ++it;
        if (it % params->check_every == 0 || it == params->max_iter) {
            // the voxel error rate of this iteration's dose (before its Adam step), and L
            CK(vamrt::launch_ver(p, dose, ddt, target, ver3, s), "voxel error rate kernels");
            CK(cudaMemcpyAsync(&host->err, p->hist + it - 1, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaMemcpyAsync(host->ver3, ver3, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
            err = host->err;
            ver = host->ver3[2] > 0 ? (double)host->ver3[0] / (double)host->ver3[2] : 0.0;
            vers[it - 1] = ver;
            if (!isfinite(err)) {
                if (report) { report->iterations = it; report->final_error = err; report->final_ver = ver; }
                return fail(VAMRT_NUMERIC, "loss is not finite at iteration %d", it);
            }
            if ((params->stop == VAMRT_STOP_VER ? ver : err) < params->tol) { converged = true; break; }
        }
    }
    if (report) {
        report->iterations = it;
        report->final_error = err;
        report->adjoint_ms = t_adj;
        report->forward_ms = t_fwd;
        report->update_ms = t_upd;
        report->final_ver = ver;
        if (report->ver_history)
            for (int i = 0; i < it; ++i) report->ver_history[i] = vers[(size_t)i];
        if (report->error_history) {
            CK(cudaMemcpyAsync(report->error_history, p->hist, sizeof(double) * it, cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
        }
    }
    return converged ? VAMRT_OK : VAMRT_NOT_CONVERGED;
}

}  // namespace

vamrt_status vamrt_optimize(vamrt_projector *p, const float *target, float *model, void *proj, void *dose,
                            const vamrt_opt_params *params, vamrt_opt_report *report, void *stream)
{
    if (!p || !target || !model || !proj || !dose || !params) return fail(VAMRT_EINVAL, "NULL argument");
    if (params->max_iter < 1 || params->max_iter > vamrt::kMaxHistory)
        return fail(VAMRT_EINVAL, "max_iter must be in 1..%d", vamrt::kMaxHistory);
    if (params->check_every < 1) return fail(VAMRT_EINVAL, "check_every must be >= 1");
    if (!(params->tol >= 0.0)) return fail(VAMRT_EINVAL, "tol must be >= 0");
    if (check_dtype(params->proj_dtype) || check_dtype(params->dose_dtype)) return VAMRT_EINVAL;
    if (params->mode != VAMRT_OPT_OBJECT && params->mode != VAMRT_OPT_PROJECTIONS && params->mode != VAMRT_OPT_GRADIENT)
        return fail(VAMRT_EINVAL, "unknown optimiser mode %d", params->mode);
    if (params->stop != VAMRT_STOP_VER && params->stop != VAMRT_STOP_ERROR)
        return fail(VAMRT_EINVAL, "unknown stop criterion %d", params->stop);
    if (params->mode == VAMRT_OPT_GRADIENT)
        return optimize_gradient(p, target, model, proj, dose, params, report, (cudaStream_t)stream);
    if (params->mode == VAMRT_OPT_PROJECTIONS && !(params->step > 0.0 && params->step <= 1.0))
        return fail(VAMRT_EINVAL, "projection-space step must be in (0, 1]");
    if (params->mode == VAMRT_OPT_OBJECT && !(params->step >= 0.0 && params->step <= 64.0))
        return fail(VAMRT_EINVAL, "object-space step must be in [0, 64] (0 = 1)");
    // object space: 0 (a zero-initialised struct) means the plain update, step 1
    const double step = params->mode == VAMRT_OPT_OBJECT && params->step == 0.0 ? 1.0 : params->step;
    if (!(params->momentum >= 0.0 && params->momentum < 1.0))
        return fail(VAMRT_EINVAL, "momentum must be in [0, 1)");
    if (params->momentum != 0.0 && (params->mode != VAMRT_OPT_OBJECT || !params->prev_model))
        return fail(VAMRT_EINVAL, "momentum needs object mode and a prev_model buffer");
    cudaStream_t s = (cudaStream_t)stream;
    double *fsum = p->red + vamrt::kRedBlocks;
    // phase timing: events ev[0..3] bracket adjoint | forward | update of one iteration
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double t_adj = 0.0, t_fwd = 0.0, t_upd = 0.0;
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() { for (int i = 0; i < 4; ++i) if (e[i]) cudaEventDestroy(e[i]); }
    } evguard{ev};
    if (params->timing)
        for (int i = 0; i < 4; ++i) CK(cudaEventCreate(&ev[i]), "cudaEventCreate");
    CK(vamrt::launch_sum(p, target, fsum, s), "target sum");
    int it = 0;
    double err = NAN, ver = NAN;
    bool converged = false;
    std::vector<double> vers((size_t)params->max_iter, NAN);
    long long *ver3 = reinterpret_cast<long long *>(p->red + vamrt::kRedBlocks + 5);
    struct Checked {
        double err;
        long long ver3[3];
    };
    Checked *host_chk = reinterpret_cast<Checked *>(p->host_err);
    const bool proj_space = params->mode == VAMRT_OPT_PROJECTIONS;
    for (; it < params->max_iter;) {
        if (params->timing) CK(cudaEventRecord(ev[0], s), "cudaEventRecord");
        if (!proj_space) {
            // g = max(0, A^T m)
            CK(vamrt::launch_pad(p, model, VAMRT_F32, s), "pad kernel");
            CK(vamrt::launch_adjoint(p, VAMRT_F32, proj, params->proj_dtype, VAMRT_CLAMP_NONNEG, s), "adjoint kernel");
        }
        if (params->timing) CK(cudaEventRecord(ev[1], s), "cudaEventRecord");
        // d = A g (left in the scratch volume), then normalise, update, error
        CK(vamrt::launch_forward(p, proj, params->proj_dtype, s), "forward kernel");
        if (params->timing) CK(cudaEventRecord(ev[2], s), "cudaEventRecord");
        CK(vamrt::launch_osmo_step(p, target, model, dose, params->dose_dtype, fsum, p->hist + it, proj_space ? 1 : 0,
                                   (float)step, (float)params->momentum,
                                   params->momentum != 0.0 ? params->prev_model : nullptr, s),
           "osmo step");
        if (proj_space) {
            // g <- max(0, g + A^T (f - dn)); the residual is in the model buffer
            CK(vamrt::launch_pad(p, model, VAMRT_F32, s), "pad kernel");
            CK(vamrt::launch_adjoint(p, VAMRT_F32, proj, params->proj_dtype, VAMRT_ACCUMULATE | VAMRT_CLAMP_NONNEG, s),
               "adjoint kernel");
        }
        if (params->timing) {
            CK(cudaEventRecord(ev[3], s), "cudaEventRecord");
            CK(cudaEventSynchronize(ev[3]), "cudaEventSynchronize");
            float ms[3];
            for (int i = 0; i < 3; ++i) CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]), "cudaEventElapsedTime");
            t_adj += ms[0];
            t_fwd += ms[1];
            t_upd += ms[2];
        }
        ++it;
        if (it % params->check_every == 0 || it == params->max_iter) {
            // the voxel error rate of this iteration's normalised dose, then E and V together
            CK(vamrt::launch_ver(p, dose, params->dose_dtype, target, ver3, s), "voxel error rate kernels");
            CK(cudaMemcpyAsync(&host_chk->err, p->hist + it - 1, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaMemcpyAsync(host_chk->ver3, ver3, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
            err = host_chk->err;
            ver = host_chk->ver3[2] > 0 ? (double)host_chk->ver3[0] / (double)host_chk->ver3[2] : 0.0;
            vers[it - 1] = ver;
            if (!isfinite(err)) {
                if (report) { report->iterations = it; report->final_error = err; report->final_ver = ver; }
                return fail(VAMRT_NUMERIC, "dose error is not finite at iteration %d (zero or NaN dose)", it);
            }
            if ((params->stop == VAMRT_STOP_VER ? ver : err) < params->tol) { converged = true; break; }
        }
    }
    if (report) {
        report->iterations = it;
        report->final_error = err;
        report->adjoint_ms = t_adj;
        report->forward_ms = t_fwd;
        report->update_ms = t_upd;
        report->final_ver = ver;
        if (report->ver_history)
            for (int i = 0; i < it; ++i) report->ver_history[i] = vers[(size_t)i];
        if (report->error_history) {
            CK(cudaMemcpyAsync(report->error_history, p->hist, sizeof(double) * it, cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
        }
    }
    return converged ? VAMRT_OK : VAMRT_NOT_CONVERGED;
}

vamrt_status vamrt_threshold_loss(vamrt_projector *p, const void *dose, vamrt_dtype dose_dtype, const float *target,
                                  double d_l, double d_h, double *loss, void *grad, vamrt_dtype grad_dtype,
                                  void *stream)
{
    if (!p || !dose || !target || !loss) return fail(VAMRT_EINVAL, "NULL argument");
    if (check_dtype(dose_dtype) || check_dtype(grad_dtype)) return VAMRT_EINVAL;
    if (!isfinite(d_l) || !isfinite(d_h)) return fail(VAMRT_EINVAL, "thresholds must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    double *scal = p->red + vamrt::kRedBlocks + 2;       // {L, 1/|P|, 1/|Q|}
    CK(vamrt::launch_threshold_loss(p, dose, dose_dtype, target, (float)d_l, (float)d_h, scal, grad, grad_dtype, s),
       "loss kernels");
    CK(cudaMemcpyAsync(loss, scal, sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    return VAMRT_OK;
}

vamrt_status vamrt_voxel_error_rate(vamrt_projector *p, const void *dose, vamrt_dtype dose_dtype, const float *target,
                                    double *ver, int32_t *threshold_index, void *stream)
{
    if (!p || !dose || !target || !ver) return fail(VAMRT_EINVAL, "NULL argument");
    if (check_dtype(dose_dtype)) return VAMRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    long long *out3 = reinterpret_cast<long long *>(p->red + vamrt::kRedBlocks + 5);
    CK(vamrt::launch_ver(p, dose, dose_dtype, target, out3, s), "voxel error rate kernels");
    long long h[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(h, out3, sizeof(h), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    *ver = h[2] > 0 ? (double)h[0] / (double)h[2] : 0.0;
    if (threshold_index) *threshold_index = (int32_t)h[1];
    return VAMRT_OK;
}

vamrt_status vamrt_conv3d_bf16(const void *x, const void *w, const float *bias, void *y, int32_t out_f32, int32_t d,
                               int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps, int32_t relu,
                               int32_t *err_flag, void *stream)
{
    if (!x || !w || !y || !err_flag) return fail(VAMRT_EINVAL, "NULL argument");
    if (d < 1 || h < 1 || wd < 1) return fail(VAMRT_EINVAL, "volume extents must be >= 1");
    if (cin < 16 || cin % 16 || cout < 16 || cout % 16 || cout > 256)
        return fail(VAMRT_EINVAL, "channels: cin a multiple of 16, cout a multiple of 16 in 16..256");
    if (taps != 1 && taps != 27) return fail(VAMRT_EINVAL, "taps must be 1 or 27");
    if (((uintptr_t)x | (uintptr_t)w | (uintptr_t)y) & 15) return fail(VAMRT_EINVAL, "x, w and y must be 16-byte aligned");
    if ((int64_t)d * h * wd * (cin > cout ? cin : cout) >= ((int64_t)1 << 40)) return fail(VAMRT_EINVAL, "too large");
    CK(vamrt::launch_conv3d_tc(x, w, bias, y, out_f32, d, h, wd, cin, cout, taps, relu, (int *)err_flag,
                               (cudaStream_t)stream),
       "conv3d kernel");
    return VAMRT_OK;
}

vamrt_status vamrt_ramlak_filter(const float *proj, float *out, int64_t rows, int32_t nu, double pixel_mm,
                                 uint32_t flags, void *stream)
{
    if (rows < 0) return fail(VAMRT_EINVAL, "rows must be >= 0");
    if (rows > 0 && (!proj || !out)) return fail(VAMRT_EINVAL, "NULL argument");
    if (nu < 1 || nu > 4096) return fail(VAMRT_EINVAL, "nu must be in 1..4096");
    if (!(pixel_mm > 0.0) || !isfinite(pixel_mm)) return fail(VAMRT_EINVAL, "pixel_mm must be positive and finite");
    if (flags & ~(uint32_t)VAMRT_CLAMP_NONNEG) return fail(VAMRT_EINVAL, "only VAMRT_CLAMP_NONNEG is accepted");
    if (((uintptr_t)proj | (uintptr_t)out) & 3) return fail(VAMRT_EINVAL, "proj and out must be 4-byte aligned");
    CK(vamrt::launch_ramlak(proj, out, rows, nu, pixel_mm, (flags & VAMRT_CLAMP_NONNEG) ? 1 : 0,
                            (cudaStream_t)stream),
       "Ram-Lak filter kernel");
    return VAMRT_OK;
}

vamrt_status vamrt_conv3d_tiling(int32_t d, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                                 int32_t *out)
{
    if (!out) return fail(VAMRT_EINVAL, "NULL argument");
    if (d < 1 || h < 1 || wd < 1 || cin < 16 || cin % 16 || cout < 16 || cout % 16 || cout > 256 ||
        (taps != 1 && taps != 27))
        return fail(VAMRT_EINVAL, "shape not accepted by vamrt_conv3d_bf16");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "device");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    vamrt::ConvHaloPlan pl;
    if (vamrt::plan_conv3d_halo(d, h, wd, cin, cout, taps, sms, &pl)) {
        out[0] = 1; out[1] = pl.TZ; out[2] = pl.TY; out[3] = pl.Nt;
    } else {
        out[0] = out[1] = out[2] = out[3] = 0;
    }
    return VAMRT_OK;
}

vamrt_status vamrt_export_u8(vamrt_projector *p, const void *proj, vamrt_dtype proj_dtype, uint8_t *codes,
                             float *dequant, double *clip, void *stream)
{
    if (!p || !proj || !codes) return fail(VAMRT_EINVAL, "NULL argument");
    if (check_dtype(proj_dtype)) return VAMRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    double *dclip = p->red + vamrt::kRedBlocks + 1;
    CK(vamrt::launch_export_u8(p, proj, proj_dtype, codes, dequant, dclip, s), "export kernels");
    if (clip) {
        CK(cudaMemcpyAsync(clip, dclip, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
    }
    return VAMRT_OK;
}

vamrt_status vamrt_copy_ray_table(const vamrt_projector *p, float *a4, float *b4, int32_t *j2)
{
    if (!p) return fail(VAMRT_EINVAL, "NULL projector");
    CK(cudaDeviceSynchronize(), "sync");
    // the table is FP64 on the device; this call hands out its FP32 rounding
    const double4_32a *src[2] = {p->tabA, p->tabB};
    float *dst[2] = {a4, b4};
    for (int t = 0; t < 2; ++t) {
        if (!dst[t]) continue;
        std::vector<double4_32a> h;
        try {
            h.resize((size_t)p->n_rays);
        } catch (...) {
            return fail(VAMRT_ENOMEM, "host allocation failed");
        }
        CK(cudaMemcpy(h.data(), src[t], sizeof(double4_32a) * p->n_rays, cudaMemcpyDeviceToHost), "copy");
        for (int64_t r = 0; r < p->n_rays; ++r) {
            dst[t][4 * r] = (float)h[r].x;
            dst[t][4 * r + 1] = (float)h[r].y;
            dst[t][4 * r + 2] = (float)h[r].z;
            dst[t][4 * r + 3] = (float)h[r].w;
        }
    }
    if (j2) CK(cudaMemcpy(j2, p->tabJ, sizeof(int2) * p->n_rays, cudaMemcpyDeviceToHost), "copy");
    return VAMRT_OK;
}

}  // extern "C"
