// Measured on-chip bandwidths of the current GPU: the denominators of the operators'
// rooflines.
//
// The operators move their per-sample data (8 trilinear corner words) through shared
// memory, and their volume boxes and dose flushes through L2, so three rates bound them:
//   - shared-memory reads: conflict-free loads from every SM with several resident
//     blocks (each warp request one 128-byte wavefront per 32 words), issued as volatile
//     loads so that none is merged, hoisted or dropped;
//   - L2 reads: 16-byte loads that bypass L1 (ld.global.cg) over a buffer that fits in L2,
//     after one pass that brings it there;
//   - L2 reductions: 16-byte vector reductions (red.global.add.v4.f32, the dose flush's
//     instruction) to distinct addresses of a buffer that fits in L2.
#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kCalThreads = 256;
constexpr int kCalWords = 4096;

__device__ __forceinline__ float lds_volatile(unsigned addr)
{
    float v;
    asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__global__ void __launch_bounds__(kCalThreads) smem_read_kernel(float *out, int iters)
{
    __shared__ float s[kCalWords];
    for (int i = threadIdx.x; i < kCalWords; i += kCalThreads) s[i] = (float)(i & 7);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // one 512-word window (16 rows of 32 banks) per warp; every load of a warp reads one
    // row, 32 distinct banks
    const unsigned base = (unsigned)__cvta_generic_to_shared(&s[(threadIdx.x >> 5) * 512 + lane]);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int it = 0; it < iters; ++it) {
        const unsigned r = (unsigned)(it & 1) * 8u;
        a0 += lds_volatile(base + 128u * (r + 0));
        a1 += lds_volatile(base + 128u * (r + 1));
        a2 += lds_volatile(base + 128u * (r + 2));
        a3 += lds_volatile(base + 128u * (r + 3));
        a0 += lds_volatile(base + 128u * (r + 4));
        a1 += lds_volatile(base + 128u * (r + 5));
        a2 += lds_volatile(base + 128u * (r + 6));
        a3 += lds_volatile(base + 128u * (r + 7));
    }
    out[blockIdx.x * kCalThreads + threadIdx.x] = a0 + a1 + a2 + a3;
}

__device__ __forceinline__ float4 ld_cg(const float4 *p)
{
    float4 v;
    asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Every thread reads 16-byte words i, i + stride, ... of buf (n4 words), `passes` times.
__global__ void __launch_bounds__(kCalThreads) l2_read_kernel(const float4 *buf, int64_t n4, int passes, float *out)
{
    const int64_t stride = (int64_t)gridDim.x * kCalThreads;
    float acc = 0.f;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = (int64_t)blockIdx.x * kCalThreads + threadIdx.x; i < n4; i += stride) {
            const float4 v = ld_cg(buf + i);
            acc += v.x + v.y + v.z + v.w;
        }
    out[blockIdx.x * kCalThreads + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(kCalThreads) l2_red_kernel(float4 *buf, int64_t n4, int passes)
{
    const int64_t stride = (int64_t)gridDim.x * kCalThreads;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = (int64_t)blockIdx.x * kCalThreads + threadIdx.x; i < n4; i += stride)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(buf + i), "f"(1.f), "f"(1.f),
                         "f"(1.f), "f"(1.f)
                         : "memory");
}

// Times `launch` (a warm-up run first) with CUDA events on s; ms <= 0 on failure.
template <class F>
float time_ms(cudaStream_t s, F launch)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = -1.f;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        launch();
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = -1.f;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return ms;
}

}  // namespace
}  // namespace vamrt

extern "C" vamrt_status vamrt_measure_smem_bandwidth(double *bytes_per_second, void *stream)
{
    if (!bytes_per_second) return VAMRT_EINVAL;
    *bytes_per_second = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VAMRT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VAMRT_ECUDA;
    const int blocks = sms * 4, iters = 1 << 15;
    float *out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * vamrt::kCalThreads) != cudaSuccess) return VAMRT_ENOMEM;
    const float ms = vamrt::time_ms(s, [&] {
        vamrt::smem_read_kernel<<<blocks, vamrt::kCalThreads, 0, s>>>(out, iters);
        vamrt::count_launches(1);
    });
    cudaFree(out);
    if (ms <= 0.f) return VAMRT_ECUDA;
    *bytes_per_second = (double)blocks * vamrt::kCalThreads * iters * 8.0 * sizeof(float) / (ms * 1e-3);
    return VAMRT_OK;
}

extern "C" vamrt_status vamrt_measure_l2_rates(double *read_bytes_per_second, double *red_ops_per_second, void *stream)
{
    if (!read_bytes_per_second || !red_ops_per_second) return VAMRT_EINVAL;
    *read_bytes_per_second = *red_ops_per_second = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VAMRT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VAMRT_ECUDA;
    // 32 MiB: resident in L2 on this part (well under its capacity)
    const int64_t n4 = (int64_t)2 * 1024 * 1024;
    const int blocks = sms * 8, passes = 16;
    float4 *buf = nullptr;
    float *out = nullptr;
    if (cudaMalloc(&buf, sizeof(float4) * n4) != cudaSuccess) return VAMRT_ENOMEM;
    if (cudaMalloc(&out, sizeof(float) * blocks * vamrt::kCalThreads) != cudaSuccess) {
        cudaFree(buf);
        return VAMRT_ENOMEM;
    }
    vamrt_status st = VAMRT_OK;
    if (cudaMemsetAsync(buf, 0, sizeof(float4) * n4, s) != cudaSuccess) st = VAMRT_ECUDA;
    if (st == VAMRT_OK) {
        const float ms = vamrt::time_ms(s, [&] {
            vamrt::l2_read_kernel<<<blocks, vamrt::kCalThreads, 0, s>>>(buf, n4, passes, out);
            vamrt::count_launches(1);
        });
        if (ms <= 0.f) st = VAMRT_ECUDA;
        else *read_bytes_per_second = (double)n4 * 16.0 * passes / (ms * 1e-3);
    }
    if (st == VAMRT_OK) {
        const float ms = vamrt::time_ms(s, [&] {
            vamrt::l2_red_kernel<<<blocks, vamrt::kCalThreads, 0, s>>>(buf, n4, passes);
            vamrt::count_launches(1);
        });
        if (ms <= 0.f) st = VAMRT_ECUDA;
        else *red_ops_per_second = (double)n4 * passes / (ms * 1e-3);
    }
    cudaFree(out);
    cudaFree(buf);
    return st;
}
