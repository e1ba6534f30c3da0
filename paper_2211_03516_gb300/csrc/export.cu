// 8-bit export of projections before the final dose simulation (Sec. 2.7: values beyond
// three standard deviations above the mean are clipped, then the range is rescaled to the
// 8-bit grey levels sent to the projector).  Reading: projections are >= 0, so only the
// upper clip applies; code = round-half-even(255 min(max(g, 0), c) / c), c = mean + 3 sigma
// (population sigma over all pixels of all angles), computed in FP64.  The dequantised
// projections code * c / 255 can be written for the final dose simulation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kEx = 256;

__device__ __forceinline__ double ldg_d(const float *p, int64_t i) { return (double)p[i]; }
__device__ __forceinline__ double ldg_d(const __nv_bfloat16 *p, int64_t i) { return (double)__bfloat162float(p[i]); }
__device__ __forceinline__ double ldg_d(const __half *p, int64_t i) { return (double)__half2float(p[i]); }

template <typename T>
__global__ void moments_kernel(const T *__restrict__ g, int64_t n, double *__restrict__ partials)
{
    __shared__ double sh[2][kEx / 32];
    double s = 0.0, s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = ldg_d(g, i);
        s += x;
        s2 += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s;
        sh[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kEx / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// clip[0] = mean + 3 sigma (fixed-order sum of the partials)
__global__ void clip_kernel(const double *__restrict__ partials, int nb, int64_t n, double *__restrict__ clip)
{
    if (threadIdx.x != 0) return;
    double s = 0.0, s2 = 0.0;
    for (int b = 0; b < nb; ++b) {
        s += partials[2 * b];
        s2 += partials[2 * b + 1];
    }
    const double mean = s / (double)n;
    const double var = fmax(s2 / (double)n - mean * mean, 0.0);
    clip[0] = mean + 3.0 * sqrt(var);
}

template <typename T>
__global__ void quantize_kernel(const T *__restrict__ g, int64_t n, const double *__restrict__ clip,
                                unsigned char *__restrict__ codes, float *__restrict__ dequant)
{
    const double c = *clip;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double q = 0.0;
        if (c > 0.0) q = rint(255.0 * fmin(fmax(ldg_d(g, i), 0.0), c) / c);   // round half to even
        codes[i] = (unsigned char)q;
        if (dequant) dequant[i] = (float)(q * c / 255.0);
    }
}

template <typename T>
cudaError_t launch_export_t(const vamrt_projector *p, const T *g, int64_t n, unsigned char *codes, float *dequant,
                            double *clip, cudaStream_t s)
{
    int64_t nb = (n + kEx - 1) / kEx;
    if (nb > kRedBlocks / 2) nb = kRedBlocks / 2;
    moments_kernel<T><<<(unsigned)nb, kEx, 0, s>>>(g, n, p->red);
    clip_kernel<<<1, 32, 0, s>>>(p->red, (int)nb, n, clip);
    unsigned gq = (unsigned)((n + kEx - 1) / kEx);
    if (gq > (unsigned)p->num_sms * 16u) gq = (unsigned)p->num_sms * 16u;
    quantize_kernel<T><<<gq, kEx, 0, s>>>(g, n, clip, codes, dequant);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_export_u8(const vamrt_projector *p, const void *proj, vamrt_dtype dt, unsigned char *codes,
                             float *dequant, double *clip, cudaStream_t s)
{
    const int64_t n = (int64_t)p->g.n_angles * p->g.nv * p->g.nu;
    if (dt == VAMRT_F32) return launch_export_t(p, (const float *)proj, n, codes, dequant, clip, s);
    if (dt == VAMRT_BF16) return launch_export_t(p, (const __nv_bfloat16 *)proj, n, codes, dequant, clip, s);
    return launch_export_t(p, (const __half *)proj, n, codes, dequant, clip, s);
}

}  // namespace vamrt
