// Ram-Lak filtering of sinogram rows for the Radon-method baseline (Sec. 2.3): the
// band-limited ramp of filtered backprojection, kernel (unit pitch) h[0] = 1/4,
// h[n] = -1 / (pi^2 n^2) for odd n, 0 for even n != 0, applied as a linear convolution
// along each row (zero outside it) and divided by the pixel pitch; optionally the
// negative values clipped to zero.  One block per row at a time: the row and the taps sit
// in shared memory, each thread forms outputs from the odd offsets only.  Memory traffic
// is one read and one write of the sinogram; the O(nu^2 / 2) multiply-adds per row bound
// the time for wide rows.
#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kRlThreads = 256;
constexpr float kInvPi2 = 0.10132118364233778f;   // 1 / pi^2

__global__ void __launch_bounds__(kRlThreads) ramlak_kernel(const float *in, float *out, int64_t rows, int nu,
                                                            float inv_tau, int clamp)
{
    extern __shared__ float sm[];
    float *row = sm;        // nu samples of the current row
    float *h = sm + nu;     // taps h[k], k = 0 .. nu - 1 (the kernel is even)
    for (int k = threadIdx.x; k < nu; k += blockDim.x)
        h[k] = k == 0 ? 0.25f : ((k & 1) ? -kInvPi2 / ((float)k * (float)k) : 0.f);
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        __syncthreads();    // the previous row's readers are done (and the taps are ready)
        for (int u = threadIdx.x; u < nu; u += blockDim.x) row[u] = in[r * nu + u];
        __syncthreads();    // the whole row is read before any output of it is written (in place)
        for (int u = threadIdx.x; u < nu; u += blockDim.x) {
            const int both = min(u, nu - 1 - u);     // offsets with a sample on either side
            float acc = 0.f;
            int k = 1;
            for (; k <= both; k += 2) acc = fmaf(h[k], row[u - k] + row[u + k], acc);
            for (; k <= u; k += 2) acc = fmaf(h[k], row[u - k], acc);
            for (; k < nu - u; k += 2) acc = fmaf(h[k], row[u + k], acc);
            float q = (0.25f * row[u] + acc) * inv_tau;
            if (clamp) q = fmaxf(q, 0.f);
            out[r * nu + u] = q;
        }
    }
}

}  // namespace

cudaError_t launch_ramlak(const float *in, float *out, int64_t rows, int nu, double pixel_mm, int clamp,
                          cudaStream_t s)
{
    if (rows == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)sms * 8;
    if (grid > rows) grid = rows;
    const size_t smem = 2 * (size_t)nu * sizeof(float);
    ramlak_kernel<<<(unsigned)grid, kRlThreads, smem, s>>>(in, out, rows, nu, (float)(1.0 / pixel_mm), clamp);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
