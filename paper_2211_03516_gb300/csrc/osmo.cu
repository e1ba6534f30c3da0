// Elementwise and reduction kernels of the projection optimiser (Sec. 2.7).
//
// Per iteration, after the two operators: the dose maximum over the resin (order-free, so
// exact), then
// one fused pass that normalises the dose, writes it out, updates the model and emits
// per-block FP64 partial sums of |dn - f|; a single block adds the partials in a fixed
// order, so the error E is deterministic.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ void st_dose(float *p, float x) { *p = x; }
__device__ __forceinline__ void st_dose(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
__device__ __forceinline__ void st_dose(__half *p, float x) { *p = __float2half_rn(x); }

template <typename T>
__device__ T block_sum(T x, T *sh)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = x;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;
}

__global__ void sum_partials_kernel(const float *__restrict__ x, int64_t n, double *__restrict__ partials)
{
    __shared__ double sh[kRedThreads / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)x[i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = scale * sum(partials[0..n)), or NaN when scale is not finite / the sum is not.
__global__ void finish_sum_kernel(const double *__restrict__ partials, int n, const double *__restrict__ divisor,
                                  double *__restrict__ out)
{
    __shared__ double sh[kRedThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = divisor ? s / *divisor : s;
}

// Maximum of the dose over the resin voxels (centres within r_inner of the axis, decided
// in FP64 without fused multiply-adds).
__global__ void resin_max_kernel(const float *__restrict__ acc, int nx, int ny, int nz, int px, int py, double h,
                                 double r2, float *__restrict__ out)
{
    const int64_t total = (int64_t)nx * ny * nz;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        const double cx = (x - 0.5 * (nx - 1)) * h, cy = (y - 0.5 * (ny - 1)) * h;
        if (__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)) > r2) continue;
        m = fmaxf(m, acc[((int64_t)(z + 1) * py + (y + 1)) * px + (x + 1)]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    // dose values are >= 0, so their bit patterns order like the values
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
}

template <typename DT>
__global__ void osmo_update_kernel(const float *__restrict__ acc, const float *__restrict__ dmax,
                                   const float *__restrict__ target, float *__restrict__ model,
                                   DT *__restrict__ dose, int nx, int ny, int nz, int px, int py,
                                   double *__restrict__ partials, int residual, float alpha, float mu,
                                   float *__restrict__ prev)
{
    __shared__ double sh[kRedThreads / 32];
    const int64_t total = (int64_t)nx * ny * nz;
    const float inv = 1.0f / *dmax;
    double err = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        const float dn = acc[((int64_t)(z + 1) * py + (y + 1)) * px + (x + 1)] * inv;
        const float f = target[i];
        st_dose(dose + i, dn);
        // object space: m <- max(0, m + alpha (f - dn) + mu (m - m_prev)) (alpha = 1, mu = 0:
        // the plain reading), m_prev <- m; projection space: the residual alpha (f - dn)
        if (residual) {
            model[i] = alpha * (f - dn);
        } else if (prev) {
            const float m = model[i];
            model[i] = fmaxf(0.f, m + alpha * (f - dn) + mu * (m - prev[i]));
            prev[i] = m;
        } else {
            model[i] = fmaxf(0.f, model[i] + alpha * (f - dn));
        }
        err += fabs((double)dn - (double)f);
    }
    const double s = block_sum(err, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

inline int red_grid(int64_t n)
{
    int64_t g = (n + kRedThreads - 1) / kRedThreads;
    if (g > kRedBlocks) g = kRedBlocks;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_sum(const vamrt_projector *p, const float *x, double *out, cudaStream_t s)
{
    const int64_t n = (int64_t)p->g.nx * p->g.ny * p->g.nz;
    const int G = red_grid(n);
    sum_partials_kernel<<<G, kRedThreads, 0, s>>>(x, n, p->red);
    finish_sum_kernel<<<1, kRedThreads, 0, s>>>(p->red, G, nullptr, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_osmo_step(const vamrt_projector *p, const float *target, float *model, void *dose,
                             vamrt_dtype dose_dt, const double *fsum, double *err_out, int residual, float alpha,
                             float mu, float *prev, cudaStream_t s)
{
    const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
    const int64_t n = (int64_t)nx * ny * nz;
    cudaError_t e = cudaMemsetAsync(p->dmax, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    int gm = (int)((n + kRedThreads - 1) / kRedThreads);
    if (gm > p->num_sms * 8) gm = p->num_sms * 8;
    const int px = p->op.px, py = p->op.py;
    resin_max_kernel<<<gm, kRedThreads, 0, s>>>(p->scratch, nx, ny, nz, px, py, p->g.voxel_mm,
                                                p->g.r_inner_mm * p->g.r_inner_mm, p->dmax);
    const int G = red_grid(n);
    if (dose_dt == VAMRT_F32)
        osmo_update_kernel<float><<<G, kRedThreads, 0, s>>>(p->scratch, p->dmax, target, model, (float *)dose,
                                                         nx, ny, nz, px, py, p->red, residual, alpha, mu, prev);
    else if (dose_dt == VAMRT_BF16)
        osmo_update_kernel<__nv_bfloat16><<<G, kRedThreads, 0, s>>>(p->scratch, p->dmax, target, model,
                                                                 (__nv_bfloat16 *)dose, nx, ny, nz, px, py, p->red, residual, alpha,
                                                                 mu, prev);
    else
        osmo_update_kernel<__half><<<G, kRedThreads, 0, s>>>(p->scratch, p->dmax, target, model, (__half *)dose, nx,
                                                          ny, nz, px, py, p->red, residual, alpha, mu, prev);
    finish_sum_kernel<<<1, kRedThreads, 0, s>>>(p->red, G, fsum, err_out);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace vamrt
