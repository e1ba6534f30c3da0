// Shared-memory read bandwidth of the current GPU, measured.
//
// The operators move their per-sample data (8 trilinear corner words) through shared
// memory, so that memory's bandwidth is the roofline they are reported against.  The
// kernel reads conflict-free 32-bit words (each warp request is one 128-byte wavefront)
// from every SM with several resident blocks, the same access width the operators use.
#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kCalThreads = 256;
constexpr int kCalWords = 4096;

// a shared-memory load the compiler may neither merge nor hoist
__device__ __forceinline__ float lds(const float *p)
{
    float v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

__global__ void __launch_bounds__(kCalThreads) smem_read_kernel(float *out, int iters, int mask)
{
    __shared__ float s[kCalWords];
    for (int i = threadIdx.x; i < kCalWords; i += kCalThreads) s[i] = (float)(i & 7);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int base = (threadIdx.x >> 5) * 512 + lane;   // one 512-word window per warp
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int it = 0; it < iters; ++it) {
        const int o = (it * 8) & mask;                     // mask = 15: rows 0..15 of the window
        a0 += lds(&s[base + 32 * ((o + 0) & 15)]);
        a1 += lds(&s[base + 32 * ((o + 1) & 15)]);
        a2 += lds(&s[base + 32 * ((o + 2) & 15)]);
        a3 += lds(&s[base + 32 * ((o + 3) & 15)]);
        a0 += lds(&s[base + 32 * ((o + 4) & 15)]);
        a1 += lds(&s[base + 32 * ((o + 5) & 15)]);
        a2 += lds(&s[base + 32 * ((o + 6) & 15)]);
        a3 += lds(&s[base + 32 * ((o + 7) & 15)]);
    }
    out[blockIdx.x * kCalThreads + threadIdx.x] = a0 + a1 + a2 + a3;
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
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    vamrt_status st = VAMRT_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = VAMRT_ECUDA;
    if (st == VAMRT_OK) {
        vamrt::smem_read_kernel<<<blocks, vamrt::kCalThreads, 0, s>>>(out, iters, 15);   // warm-up
        cudaEventRecord(e0, s);
        vamrt::smem_read_kernel<<<blocks, vamrt::kCalThreads, 0, s>>>(out, iters, 15);
        cudaEventRecord(e1, s);
        vamrt::count_launches(2);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
            st = VAMRT_ECUDA;
        else
            *bytes_per_second = (double)blocks * vamrt::kCalThreads * iters * 8.0 * sizeof(float) / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
