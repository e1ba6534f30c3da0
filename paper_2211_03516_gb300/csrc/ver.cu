// Voxel error rate of a dose against a binary target: the fraction of resin voxels whose
// printed state (dose above a threshold) differs from the target, at the best of 1023
// thresholds tau_i = (i / 1024) max(dose), i = 1..1023, the maximum taken over the resin.  It measures how well a dose
// prints the part independently of the dose's scale, the quantity the optimiser's
// stopping rule is after (Sec. 2.7).
//
// Exact integer bookkeeping: each resin voxel falls in bin b = min(floor(x * (1024/max)),
// 1023) (FP32, the dose's precision), so "x >= tau_i" is "b >= i"; two 1024-bin histograms
// (in-part, out-of-part) give every threshold's mismatch count by prefix sums.  Resin =
// voxel centres within r_inner of the axis (decided in FP64).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kBins = 1024;
constexpr int kVerThreads = 256;

__device__ __forceinline__ float ldd(const float *p) { return *p; }
__device__ __forceinline__ float ldd(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldd(const __half *p) { return __half2float(*p); }

// maximum over the resin voxels (the same FP64 test as the histogram below)
template <typename DT>
__global__ void dose_max_kernel(const DT *__restrict__ dose, int nx, int ny, int nz, double h, double r2,
                                float *__restrict__ out)
{
    const int64_t n = (int64_t)nx * ny * nz;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny);
        const double cx = (x - 0.5 * (nx - 1)) * h, cy = (y - 0.5 * (ny - 1)) * h;
        if (__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)) > r2) continue;
        m = fmaxf(m, ldd(dose + i));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));   // m >= 0
}

// hist[0..1023]: in-part, hist[1024..2047]: out-of-part (resin voxels only)
template <typename DT>
__global__ void ver_hist_kernel(const DT *__restrict__ dose, const float *__restrict__ target, int nx, int ny,
                                int nz, double h, double r2, const float *__restrict__ dmax,
                                unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[2 * kBins];
    for (int i = threadIdx.x; i < 2 * kBins; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const float m = *dmax;
    const float scale = m > 0.f ? (float)kBins / m : 0.f;   // all-zero dose: every voxel in bin 0
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny);
        const double cx = (x - 0.5 * (nx - 1)) * h, cy = (y - 0.5 * (ny - 1)) * h;
        if (__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)) > r2) continue;   // no FMA: plain FP64 rounding
        const float q = ldd(dose + i) * scale;
        int b = (int)floorf(q);
        b = min(max(b, 0), kBins - 1);
        atomicAdd(&sh[(target[i] > 0.5f ? 0 : kBins) + b], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kBins; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// out[0] = best mismatch count, out[1] = best threshold index, out[2] = resin voxel count
__global__ void ver_scan_kernel(const unsigned *__restrict__ hist, long long *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    long long in_below = 0, out_total = 0, in_total = 0;
    for (int b = 0; b < kBins; ++b) {
        in_total += hist[b];
        out_total += hist[kBins + b];
    }
    long long out_below = 0, best = -1, best_i = 1;
    for (int i = 1; i < kBins; ++i) {
        in_below += hist[i - 1];
        out_below += hist[kBins + i - 1];
        const long long mis = in_below + (out_total - out_below);
        if (best < 0 || mis < best) {
            best = mis;
            best_i = i;
        }
    }
    out[0] = best;
    out[1] = best_i;
    out[2] = in_total + out_total;
}

}  // namespace

cudaError_t launch_ver(const vamrt_projector *p, const void *dose, vamrt_dtype dt, const float *target,
                       long long *out3, cudaStream_t s)
{
    const int nx = p->g.nx, ny = p->g.ny, nz = p->g.nz;
    const int64_t n = (int64_t)nx * ny * nz;
    unsigned *hist = reinterpret_cast<unsigned *>(p->red);   // 2 x 1024 counters (8 KB)
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned) * 2 * kBins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->dmax, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    unsigned g = (unsigned)((n + kVerThreads - 1) / kVerThreads);
    if (g > (unsigned)p->num_sms * 8u) g = (unsigned)p->num_sms * 8u;
    const double r2 = p->g.r_inner_mm * p->g.r_inner_mm;
    if (dt == VAMRT_F32) {
        dose_max_kernel<float><<<g, kVerThreads, 0, s>>>((const float *)dose, nx, ny, nz, p->g.voxel_mm, r2,
                                                          p->dmax);
        ver_hist_kernel<float><<<g, kVerThreads, 0, s>>>((const float *)dose, target, nx, ny, nz, p->g.voxel_mm, r2,
                                                          p->dmax, hist);
    } else if (dt == VAMRT_F16) {
        dose_max_kernel<__half><<<g, kVerThreads, 0, s>>>((const __half *)dose, nx, ny, nz, p->g.voxel_mm, r2, p->dmax);
        ver_hist_kernel<__half><<<g, kVerThreads, 0, s>>>((const __half *)dose, target, nx, ny, nz, p->g.voxel_mm, r2,
                                                           p->dmax, hist);
    } else {
        dose_max_kernel<__nv_bfloat16><<<g, kVerThreads, 0, s>>>((const __nv_bfloat16 *)dose, nx, ny, nz,
                                                                  p->g.voxel_mm, r2, p->dmax);
        ver_hist_kernel<__nv_bfloat16><<<g, kVerThreads, 0, s>>>((const __nv_bfloat16 *)dose, target, nx, ny, nz,
                                                                  p->g.voxel_mm, r2, p->dmax, hist);
    }
    ver_scan_kernel<<<1, 32, 0, s>>>(hist, out3);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace vamrt
