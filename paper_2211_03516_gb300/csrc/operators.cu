// The two hot operators: projection (adjoint, gather) and dose (forward, scatter).
//
// Work mapping (both operators): one thread per pixel and angle; the 32 lanes of a warp
// are 32 adjacent pixels u of one row v, so at every step their samples lie side by
// side in the volume and their voxel fetches / reductions fall in few cache lines.  A
// block is 32 x 4 pixels of one angle; blocks of one angle are launched together so the
// volume region they sweep stays resident in L1/L2.  Each thread walks the aperture
// samples of its pixel in turn and, along each ray, the midpoint samples
// s_j = (j + 1/2) delta.  Per ray, the entry point and direction are rotated into the
// vial frame once (FP32), so a sample costs three FMAs for its position, one exp2 for
// Beer-Lambert, the trilinear weights (Sec. 2.2) and 8 voxel accesses.
//
// The caller's volume is first copied into a scratch volume with one voxel of zero halo,
// which removes every per-corner bounds test from the inner loop (zero padding outside
// the grid); index clamps remain only as a guard that never binds for valid geometry.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace vamrt {
namespace {

__device__ __forceinline__ float ld_val(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p)
{
    const unsigned short raw = __ldg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float(((unsigned)raw) << 16);
}
__device__ __forceinline__ void st_val(float *p, float x) { *p = x; }
__device__ __forceinline__ void st_val(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
__device__ __forceinline__ float ld_plain(const float *p) { return *p; }
__device__ __forceinline__ float ld_plain(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// ---------------------------------------------------------------------------------
// halo copy: scratch[zp][yp][xp] = vol[zp-1][yp-1][xp-1] inside, 0 on the halo
// ---------------------------------------------------------------------------------
template <typename VT>
__global__ void pad_kernel(const VT *__restrict__ vol, VT *__restrict__ out, int nx, int ny, int nz,
                           int64_t total)
{
    const int px = nx + 2, py = ny + 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int xp = (int)(i % px);
        const int yp = (int)((i / px) % py);
        const int zp = (int)(i / ((int64_t)px * py));
        VT val = VT(0.0f);
        if (xp >= 1 && xp <= nx && yp >= 1 && yp <= ny && zp >= 1 && zp <= nz)
            val = vol[((int64_t)(zp - 1) * ny + (yp - 1)) * nx + (xp - 1)];
        out[i] = val;
    }
}

// dose[z][y][x] (+)= scratch[z+1][y+1][x+1]
template <typename DT>
__global__ void unpad_kernel(const float *__restrict__ acc, DT *__restrict__ dose, int nx, int ny, int nz,
                             int accumulate)
{
    const int64_t total = (int64_t)nx * ny * nz;
    const int px = nx + 2, py = ny + 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        float val = acc[((int64_t)(z + 1) * py + (y + 1)) * px + (x + 1)];
        if (accumulate) val += ld_plain(dose + i);
        st_val(dose + i, val);
    }
}

// Per-ray setup shared by both operators: rotated entry point and per-sample step in
// padded index coordinates, and the log2 attenuation per sample.
struct RaySetup {
    float qx, qy, qz;     // position of "sample -1/2" (the entry point)
    float sx, sy, sz;     // advance per sample
    float att;            // log2 of the Beer-Lambert factor per sample
};

__device__ __forceinline__ RaySetup ray_setup(const OpParams &P, float4 A, float4 B, float2 cs)
{
    RaySetup R;
    R.qx = P.cx + (cs.x * A.x - cs.y * A.y);
    R.qy = P.cy + (cs.y * A.x + cs.x * A.y);
    R.qz = P.cz + A.z;
    R.sx = (cs.x * B.x - cs.y * B.y) * A.w;
    R.sy = (cs.y * B.x + cs.x * B.y) * A.w;
    R.sz = B.z * A.w;
    R.att = P.neg_mu_vox_log2e * A.w;
    return R;
}

struct Cell {
    int base;             // linear padded index of corner (0,0,0)
    float fx, fy, fz;     // fractional position inside the cell
};

__device__ __forceinline__ Cell locate(const OpParams &P, float qx, float qy, float qz)
{
    const float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
    Cell c;
    c.fx = qx - flx;
    c.fy = qy - fly;
    c.fz = qz - flz;
    const int ix = min(max((int)flx, 0), P.px - 2);
    const int iy = min(max((int)fly, 0), P.py - 2);
    const int iz = min(max((int)flz, 0), P.pz - 2);
    c.base = (iz * P.py + iy) * P.px + ix;
    return c;
}

// ---------------------------------------------------------------------------------
// projection (adjoint): proj[k][v][u] = sum_a W_a sum_j exp(-mu s_j) trilinear(vol, x_j)
// ---------------------------------------------------------------------------------
template <typename VT, typename PT>
__global__ void __launch_bounds__(128) adjoint_kernel(OpParams P, const VT *__restrict__ vol,
                                                      PT *__restrict__ proj, uint32_t flags)
{
    const int u = blockIdx.x * 32 + threadIdx.x;
    const int v = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z;
    if (u >= P.nu || v >= P.nv) return;
    const float2 cs = P.cs[k];
    const int sxy = P.px * P.py;
    float acc = 0.f;
    for (int a = 0; a < P.M; ++a) {
        const int64_t r = ((int64_t)a * P.nv + v) * P.nu + u;
        const int2 J = P.J[r];
        if (J.x >= J.y) continue;
        const RaySetup R = ray_setup(P, P.A[r], P.B[r], cs);
        float ray = 0.f;
        for (int j = J.x; j < J.y; ++j) {
            const float t = (float)j + 0.5f;
            const Cell c = locate(P, fmaf(t, R.sx, R.qx), fmaf(t, R.sy, R.qy), fmaf(t, R.sz, R.qz));
            const VT *p = vol + c.base;
            const float v000 = ld_val(p), v100 = ld_val(p + 1);
            const float v010 = ld_val(p + P.px), v110 = ld_val(p + P.px + 1);
            const float v001 = ld_val(p + sxy), v101 = ld_val(p + sxy + 1);
            const float v011 = ld_val(p + sxy + P.px), v111 = ld_val(p + sxy + P.px + 1);
            const float x00 = fmaf(c.fx, v100 - v000, v000);
            const float x10 = fmaf(c.fx, v110 - v010, v010);
            const float x01 = fmaf(c.fx, v101 - v001, v001);
            const float x11 = fmaf(c.fx, v111 - v011, v011);
            const float y0 = fmaf(c.fy, x10 - x00, x00);
            const float y1 = fmaf(c.fy, x11 - x01, x01);
            const float val = fmaf(c.fz, y1 - y0, y0);
            ray = fmaf(exp2f(t * R.att), val, ray);
        }
        acc = fmaf(P.B[r].w, ray, acc);
    }
    PT *out = proj + ((int64_t)k * P.nv + v) * P.nu + u;
    if (flags & VAMRT_ACCUMULATE) acc += ld_plain(out);
    if (flags & VAMRT_CLAMP_NONNEG) acc = fmaxf(acc, 0.f);
    st_val(out, acc);
}

// ---------------------------------------------------------------------------------
// dose (forward): scratch[corner] += proj[k][v][u] W_a exp(-mu s_j) w_corner
// ---------------------------------------------------------------------------------
template <typename PT>
__global__ void __launch_bounds__(128) forward_kernel(OpParams P, const PT *__restrict__ proj,
                                                      float *__restrict__ acc)
{
    const int u = blockIdx.x * 32 + threadIdx.x;
    const int v = blockIdx.y * 4 + threadIdx.y;
    const int k = blockIdx.z;
    if (u >= P.nu || v >= P.nv) return;
    const float g = ld_plain(proj + ((int64_t)k * P.nv + v) * P.nu + u);
    if (g == 0.f) return;                      // adds exactly zero
    const float2 cs = P.cs[k];
    const int sxy = P.px * P.py;
    for (int a = 0; a < P.M; ++a) {
        const int64_t r = ((int64_t)a * P.nv + v) * P.nu + u;
        const int2 J = P.J[r];
        if (J.x >= J.y) continue;
        const RaySetup R = ray_setup(P, P.A[r], P.B[r], cs);
        const float gw = g * P.B[r].w;
        for (int j = J.x; j < J.y; ++j) {
            const float t = (float)j + 0.5f;
            const Cell c = locate(P, fmaf(t, R.sx, R.qx), fmaf(t, R.sy, R.qy), fmaf(t, R.sz, R.qz));
            const float w = gw * exp2f(t * R.att);
            const float wz1 = w * c.fz, wz0 = w - wz1;
            const float w01 = wz0 * c.fy, w00 = wz0 - w01;
            const float w11 = wz1 * c.fy, w10 = wz1 - w11;
            float *p = acc + c.base;
            atomicAdd(p, w00 - w00 * c.fx);
            atomicAdd(p + 1, w00 * c.fx);
            atomicAdd(p + P.px, w01 - w01 * c.fx);
            atomicAdd(p + P.px + 1, w01 * c.fx);
            atomicAdd(p + sxy, w10 - w10 * c.fx);
            atomicAdd(p + sxy + 1, w10 * c.fx);
            atomicAdd(p + sxy + P.px, w11 - w11 * c.fx);
            atomicAdd(p + sxy + P.px + 1, w11 * c.fx);
        }
    }
}

inline unsigned grid_for(const vamrt_projector *p, int64_t n, int threads)
{
    int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)p->num_sms * 16;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (unsigned)want;
}

inline dim3 op_grid(const OpParams &P) { return dim3((P.nu + 31) / 32, (P.nv + 3) / 4, P.n_angles); }

}  // namespace

cudaError_t launch_pad(const vamrt_projector *p, const void *vol, vamrt_dtype dt, cudaStream_t s)
{
    const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
    const unsigned grid = grid_for(p, p->pad_elems, 256);
    if (dt == VAMRT_F32)
        pad_kernel<float><<<grid, 256, 0, s>>>((const float *)vol, p->scratch, nx, ny, nz, p->pad_elems);
    else
        pad_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)vol,
                                                       (__nv_bfloat16 *)p->scratch, nx, ny, nz, p->pad_elems);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const vamrt_projector *p, vamrt_dtype vol_dt, void *proj, vamrt_dtype proj_dt,
                           uint32_t flags, cudaStream_t s)
{
    const dim3 grid = op_grid(p->op), block(32, 4);
    if (vol_dt == VAMRT_F32) {
        if (proj_dt == VAMRT_F32)
            adjoint_kernel<float, float><<<grid, block, 0, s>>>(p->op, p->scratch, (float *)proj, flags);
        else
            adjoint_kernel<float, __nv_bfloat16><<<grid, block, 0, s>>>(p->op, p->scratch,
                                                                        (__nv_bfloat16 *)proj, flags);
    } else {
        const __nv_bfloat16 *vol = (const __nv_bfloat16 *)p->scratch;
        if (proj_dt == VAMRT_F32)
            adjoint_kernel<__nv_bfloat16, float><<<grid, block, 0, s>>>(p->op, vol, (float *)proj, flags);
        else
            adjoint_kernel<__nv_bfloat16, __nv_bfloat16><<<grid, block, 0, s>>>(p->op, vol,
                                                                                (__nv_bfloat16 *)proj, flags);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_forward(const vamrt_projector *p, const void *proj, vamrt_dtype proj_dt, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p->scratch, 0, sizeof(float) * p->pad_elems, s);
    if (e != cudaSuccess) return e;
    const dim3 grid = op_grid(p->op), block(32, 4);
    if (proj_dt == VAMRT_F32)
        forward_kernel<float><<<grid, block, 0, s>>>(p->op, (const float *)proj, p->scratch);
    else
        forward_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(p->op, (const __nv_bfloat16 *)proj, p->scratch);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unpad(const vamrt_projector *p, void *dose, vamrt_dtype dt, uint32_t flags, cudaStream_t s)
{
    const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
    const unsigned grid = grid_for(p, (int64_t)nx * ny * nz, 256);
    const int accumulate = (flags & VAMRT_ACCUMULATE) ? 1 : 0;
    if (dt == VAMRT_F32)
        unpad_kernel<float><<<grid, 256, 0, s>>>(p->scratch, (float *)dose, nx, ny, nz, accumulate);
    else
        unpad_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(p->scratch, (__nv_bfloat16 *)dose, nx, ny, nz,
                                                         accumulate);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
