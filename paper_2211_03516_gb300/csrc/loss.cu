// Thresholded dose loss and its gradient (the differentiable path around the dose
// operator; the paper's optimiser works on the same in-part / out-of-part dose contrast):
//   L(D) = (1/|P|) sum_{v in P} relu(d_h - D_v)^2 + (1/|Q|) sum_{v in Q} relu(D_v - d_l)^2,
//   P = {target > 1/2}, Q = the other voxels;
//   dL/dD_v = -2 relu(d_h - D_v) / |P| on P,  +2 relu(D_v - d_l) / |Q| on Q.
// Three launches: per-block FP64 partial sums (counts and squared violations), one block
// that adds them in a fixed order (deterministic L), and the elementwise gradient.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kLossThreads = 256;

__device__ __forceinline__ float ldv(const float *p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stv(float *p, float x) { *p = x; }
__device__ __forceinline__ void stv(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
__device__ __forceinline__ float ldv(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void stv(__half *p, float x) { *p = __float2half_rn(x); }

__device__ double block_sum_d(double x, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;
}

// partials[4 b + {0,1,2,3}] = (|P| count, sum_P relu(d_h - D)^2, |Q| count, sum_Q relu(D - d_l)^2)
template <typename DT>
__global__ void loss_partials_kernel(const DT *__restrict__ dose, const float *__restrict__ target, int64_t n,
                                     float d_l, float d_h, double *__restrict__ partials)
{
    __shared__ double sh[kLossThreads / 32];
    double np = 0.0, sp = 0.0, nq = 0.0, sq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float D = ldv(dose + i);
        if (target[i] > 0.5f) {
            const double r = fmax((double)d_h - (double)D, 0.0);
            np += 1.0;
            sp += r * r;
        } else {
            const double r = fmax((double)D - (double)d_l, 0.0);
            nq += 1.0;
            sq += r * r;
        }
    }
    const double a = block_sum_d(np, sh), b = block_sum_d(sp, sh), c = block_sum_d(nq, sh), d = block_sum_d(sq, sh);
    if (threadIdx.x == 0) {
        partials[4 * blockIdx.x + 0] = a;
        partials[4 * blockIdx.x + 1] = b;
        partials[4 * blockIdx.x + 2] = c;
        partials[4 * blockIdx.x + 3] = d;
    }
}

// out[0] = L, out[1] = 1/max(|P|,1), out[2] = 1/max(|Q|,1)
__global__ void loss_finish_kernel(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    __shared__ double sh[kLossThreads / 32];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int k = 0; k < 4; ++k) s[k] += partials[4 * b + k];
    double t[4];
    for (int k = 0; k < 4; ++k) t[k] = block_sum_d(s[k], sh);
    if (threadIdx.x == 0) {
        const double ip = 1.0 / fmax(t[0], 1.0), iq = 1.0 / fmax(t[2], 1.0);
        out[0] = t[1] * ip + t[3] * iq;
        out[1] = ip;
        out[2] = iq;
    }
}

template <typename DT, typename GT>
__global__ void loss_grad_kernel(const DT *__restrict__ dose, const float *__restrict__ target, int64_t n, float d_l,
                                 float d_h, const double *__restrict__ scal, GT *__restrict__ grad)
{
    const float ip = (float)scal[1], iq = (float)scal[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float D = ldv(dose + i);
        const float g = target[i] > 0.5f ? -2.0f * fmaxf(d_h - D, 0.f) * ip : 2.0f * fmaxf(D - d_l, 0.f) * iq;
        stv(grad + i, g);
    }
}

template <typename DT>
cudaError_t launch_loss_t(const vamrt_projector *p, const DT *dose, const float *target, float d_l, float d_h,
                          double *loss3, void *grad, vamrt_dtype grad_dt, cudaStream_t s)
{
    const int64_t n = (int64_t)p->g.nx * p->g.ny * p->g.nz;
    int64_t nb = (n + kLossThreads - 1) / kLossThreads;
    if (nb > kRedBlocks / 4) nb = kRedBlocks / 4;
    loss_partials_kernel<DT><<<(unsigned)nb, kLossThreads, 0, s>>>(dose, target, n, d_l, d_h, p->red);
    loss_finish_kernel<<<1, kLossThreads, 0, s>>>(p->red, (int)nb, loss3);
    unsigned g = (unsigned)((n + kLossThreads - 1) / kLossThreads);
    if (g > (unsigned)p->num_sms * 16u) g = (unsigned)p->num_sms * 16u;
    if (grad) {
        if (grad_dt == VAMRT_F32)
            loss_grad_kernel<DT, float><<<g, kLossThreads, 0, s>>>(dose, target, n, d_l, d_h, loss3, (float *)grad);
        else if (grad_dt == VAMRT_BF16)
            loss_grad_kernel<DT, __nv_bfloat16><<<g, kLossThreads, 0, s>>>(dose, target, n, d_l, d_h, loss3,
                                                                           (__nv_bfloat16 *)grad);
        else
            loss_grad_kernel<DT, __half><<<g, kLossThreads, 0, s>>>(dose, target, n, d_l, d_h, loss3, (__half *)grad);
        count_launches(1);
    }
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_threshold_loss(const vamrt_projector *p, const void *dose, vamrt_dtype dose_dt,
                                  const float *target, float d_l, float d_h, double *loss3, void *grad,
                                  vamrt_dtype grad_dt, cudaStream_t s)
{
    if (dose_dt == VAMRT_F32)
        return launch_loss_t(p, (const float *)dose, target, d_l, d_h, loss3, grad, grad_dt, s);
    if (dose_dt == VAMRT_BF16)
        return launch_loss_t(p, (const __nv_bfloat16 *)dose, target, d_l, d_h, loss3, grad, grad_dt, s);
    return launch_loss_t(p, (const __half *)dose, target, d_l, d_h, loss3, grad, grad_dt, s);
}

// ---- the gradient optimiser's normalisations ------------------------------------------
namespace {

// partials[2 b + {0, 1}] = (count, sum) of x over the elements selected by target > 1/2
// (target given) or by x > 0 (target NULL)
template <typename T>
__global__ void masked_sum_kernel(const T *__restrict__ x, const float *__restrict__ target, int64_t n,
                                  double *__restrict__ partials)
{
    __shared__ double sh[kLossThreads / 32];
    double c = 0.0, t = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float xi = ldv(x + i);
        if (target ? target[i] > 0.5f : xi > 0.f) {
            c += 1.0;
            t += (double)xi;
        }
    }
    const double a = block_sum_d(c, sh), b = block_sum_d(t, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// out[0] = count, out[1] = sum, added in a fixed order
__global__ void masked_sum_finish_kernel(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    __shared__ double sh[kLossThreads / 32];
    double c = 0.0, t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        c += partials[2 * b];
        t += partials[2 * b + 1];
    }
    const double a = block_sum_d(c, sh), b = block_sum_d(t, sh);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// master = s x (FP32), and the storage copy of it when x is not the master itself
template <typename T>
__global__ void scale_master_kernel(T *__restrict__ x, float *__restrict__ master, int64_t n, float s)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float m = s * ldv(x + i);
        master[i] = m;
        if ((void *)x != (void *)master) stv(x + i, m);
    }
}

template <typename T>
cudaError_t masked_sum_t(const vamrt_projector *p, const T *x, const float *target, int64_t n, double *out2,
                         cudaStream_t s)
{
    int64_t nb = (n + kLossThreads - 1) / kLossThreads;
    if (nb > kRedBlocks / 2) nb = kRedBlocks / 2;
    if (nb < 1) nb = 1;
    masked_sum_kernel<T><<<(unsigned)nb, kLossThreads, 0, s>>>(x, target, n, p->red);
    masked_sum_finish_kernel<<<1, kLossThreads, 0, s>>>(p->red, (int)nb, out2);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_masked_sum(const vamrt_projector *p, const void *x, vamrt_dtype dt, const float *target,
                              int64_t n, double *out2, cudaStream_t s)
{
    if (dt == VAMRT_F32) return masked_sum_t(p, (const float *)x, target, n, out2, s);
    if (dt == VAMRT_BF16) return masked_sum_t(p, (const __nv_bfloat16 *)x, target, n, out2, s);
    return masked_sum_t(p, (const __half *)x, target, n, out2, s);
}

cudaError_t launch_scale_master(const vamrt_projector *p, void *x, vamrt_dtype dt, float *master, int64_t n, float sc,
                                cudaStream_t s)
{
    unsigned g = (unsigned)((n + kLossThreads - 1) / kLossThreads);
    if (g > (unsigned)p->num_sms * 16u) g = (unsigned)p->num_sms * 16u;
    if (g < 1) g = 1;
    if (dt == VAMRT_F32)
        scale_master_kernel<float><<<g, kLossThreads, 0, s>>>((float *)x, master, n, sc);
    else if (dt == VAMRT_BF16)
        scale_master_kernel<__nv_bfloat16><<<g, kLossThreads, 0, s>>>((__nv_bfloat16 *)x, master, n, sc);
    else
        scale_master_kernel<__half><<<g, kLossThreads, 0, s>>>((__half *)x, master, n, sc);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
