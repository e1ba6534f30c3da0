// Layout, elementwise and optimiser kernels of the warm-start network (everything
// around its tensor-core convolutions).  Activations are channels-last BF16
// [D][H][W][C]; master weights and optimiser moments are FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <math.h>

#include "internal.cuh"

namespace vamrt {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ __nv_bfloat16 tobf(float v) { return __float2bfloat16_rn(v); }

inline unsigned grid_n(int64_t n)
{
    int64_t g = (n + kT - 1) / kT;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

inline bool aligned16(const void *p, const void *q) { return (((uintptr_t)p | (uintptr_t)q) & 15) == 0; }

#define GRID_STRIDE(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// fine grid [D][H][W][C] <-> coarse grid [D/2][H/2][W/2][C]
__global__ void avgpool2_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, int D, int H,
                                int W, int C)
{
    const int d = D / 2, h = H / 2, w = W / 2;
    const int64_t n = (int64_t)d * h * w * C;
    GRID_STRIDE(i, n)
    {
        const int c = (int)(i % C);
        const int64_t q = i / C;
        const int x = (int)(q % w), y = (int)((q / w) % h), z = (int)(q / ((int64_t)w * h));
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
            s += bf(in[(((int64_t)zz * H + yy) * W + xx) * C + c]);
        }
        out[i] = tobf(0.125f * s);
    }
}

// ---- 16-byte variants: eight channels per thread (C a multiple of 8, 16-byte aligned
// pointers), the same per-element arithmetic in the same order as the scalar kernels, so
// bit-identical results with one vector load / store instead of eight scalar ones ----
__device__ __forceinline__ void unpack8(const uint4 v, float f[8])
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float f[8])
{
    uint4 v;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return v;
}

// op 0: average pool (scale 0.125), op 3: sum of 8 (scale 1); G = C / 8 groups
__global__ void pool8_kernel(const uint4 *__restrict__ in, uint4 *__restrict__ out, int D, int H, int W, int G,
                             float scale)
{
    const int d = D / 2, h = H / 2, w = W / 2;
    const int64_t n = (int64_t)d * h * w * G;
    GRID_STRIDE(i, n)
    {
        const int g = (int)(i % G);
        const int64_t q = i / G;
        const int x = (int)(q % w), y = (int)((q / w) % h), z = (int)(q / ((int64_t)w * h));
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
            float f[8];
            unpack8(in[(((int64_t)zz * H + yy) * W + xx) * G + g], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += f[e];
        }
        if (scale != 1.f) {
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] = scale * s[e];
        }
        out[i] = pack8(s);
    }
}

// fine voxel <- scale x its coarse voxel (scale 1: nearest upsample; 1/8: pool backward)
__global__ void spread8_kernel(const uint4 *__restrict__ coarse, uint4 *__restrict__ fine, int D, int H, int W, int G,
                               float scale)
{
    const int64_t n = (int64_t)D * H * W * G;
    const int h = H / 2, w = W / 2;
    GRID_STRIDE(i, n)
    {
        const int g = (int)(i % G);
        const int64_t q = i / G;
        const int x = (int)(q % W), y = (int)((q / W) % H), z = (int)(q / ((int64_t)W * H));
        const uint4 v = coarse[(((int64_t)(z / 2) * h + y / 2) * w + x / 2) * G + g];
        if (scale == 1.f) {
            fine[i] = v;
        } else {
            float f[8];
            unpack8(v, f);
#pragma unroll
            for (int e = 0; e < 8; ++e) f[e] = scale * f[e];
            fine[i] = pack8(f);
        }
    }
}

__global__ void concat8_kernel(const uint4 *__restrict__ a, int ga, const uint4 *__restrict__ b, int gb,
                               uint4 *__restrict__ out, int64_t npos, int backward)
{
    const int G = ga + gb;
    GRID_STRIDE(i, npos * G)
    {
        const int g = (int)(i % G);
        const int64_t p = i / G;
        if (!backward)
            out[i] = g < ga ? a[p * ga + g] : b[p * gb + (g - ga)];
        else if (g < ga)
            const_cast<uint4 *>(a)[p * ga + g] = out[i];
        else
            const_cast<uint4 *>(b)[p * gb + (g - ga)] = out[i];
    }
}

__global__ void relu_bwd8_kernel(const uint4 *__restrict__ y, uint4 *__restrict__ dy, int64_t n8)
{
    GRID_STRIDE(i, n8)
    {
        float fy[8], fd[8];
        unpack8(y[i], fy);
        const uint4 d = dy[i];
        unpack8(d, fd);
        bool any = false;
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (!(fy[e] > 0.f)) { fd[e] = 0.f; any = true; }
        if (any) dy[i] = pack8(fd);
    }
}

// db[c] += sum_p dy[p][c], 256 / G positions per block step (G = C / 8 divides 256).  A
// few blocks per SM, each streaming many positions with four loads in flight per thread:
// every block ends in C same-address global atomics, which serialise in L2.
__global__ void bias_grad8_kernel(const uint4 *__restrict__ dy, float *__restrict__ db, int64_t npos, int G)
{
    __shared__ float acc[256];
    const int C = 8 * G, per = kT / G, g = threadIdx.x % G, p0 = threadIdx.x / G;
    for (int c = threadIdx.x; c < C; c += blockDim.x) acc[c] = 0.f;
    __syncthreads();
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int64_t step = (int64_t)gridDim.x * per;
    int64_t p = (int64_t)blockIdx.x * per + p0;
    for (; p + 3 * step < npos; p += 4 * step) {
        uint4 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = dy[(p + k * step) * G + g];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float f[8];
            unpack8(q[k], f);
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += f[e];
        }
    }
    for (; p < npos; p += step) {
        float f[8];
        unpack8(dy[p * G + g], f);
#pragma unroll
        for (int e = 0; e < 8; ++e) s[e] += f[e];
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) atomicAdd(&acc[8 * g + e], s[e]);
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], acc[c]);
}

// mode 0: average-pool backward (each fine voxel gets coarse / 8)
// mode 1: nearest upsample (each fine voxel gets its coarse voxel)
__global__ void spread2_kernel(const __nv_bfloat16 *__restrict__ coarse, __nv_bfloat16 *__restrict__ fine, int D,
                               int H, int W, int C, float scale)
{
    const int64_t n = (int64_t)D * H * W * C;
    const int h = H / 2, w = W / 2;
    GRID_STRIDE(i, n)
    {
        const int c = (int)(i % C);
        const int64_t q = i / C;
        const int x = (int)(q % W), y = (int)((q / W) % H), z = (int)(q / ((int64_t)W * H));
        fine[i] = tobf(scale * bf(coarse[(((int64_t)(z / 2) * h + y / 2) * w + x / 2) * C + c]));
    }
}

// nearest-upsample backward: coarse = sum of its 8 fine voxels
__global__ void sum2_kernel(const __nv_bfloat16 *__restrict__ fine, __nv_bfloat16 *__restrict__ coarse, int D, int H,
                            int W, int C)
{
    const int d = D / 2, h = H / 2, w = W / 2;
    const int64_t n = (int64_t)d * h * w * C;
    GRID_STRIDE(i, n)
    {
        const int c = (int)(i % C);
        const int64_t q = i / C;
        const int x = (int)(q % w), y = (int)((q / w) % h), z = (int)(q / ((int64_t)w * h));
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
            s += bf(fine[(((int64_t)zz * H + yy) * W + xx) * C + c]);
        }
        coarse[i] = tobf(s);
    }
}

__global__ void concat_kernel(const __nv_bfloat16 *__restrict__ a, int ca, const __nv_bfloat16 *__restrict__ b, int cb,
                              __nv_bfloat16 *__restrict__ out, int64_t npos)
{
    const int C = ca + cb;
    GRID_STRIDE(i, npos * C)
    {
        const int c = (int)(i % C);
        const int64_t p = i / C;
        out[i] = c < ca ? a[p * ca + c] : b[p * cb + (c - ca)];
    }
}

__global__ void split_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ a, int ca,
                             __nv_bfloat16 *__restrict__ b, int cb, int64_t npos)
{
    const int C = ca + cb;
    GRID_STRIDE(i, npos * C)
    {
        const int c = (int)(i % C);
        const int64_t p = i / C;
        if (c < ca)
            a[p * ca + c] = in[i];
        else
            b[p * cb + (c - ca)] = in[i];
    }
}

// dy <- dy where y > 0, else 0
__global__ void relu_bwd_kernel(const __nv_bfloat16 *__restrict__ y, __nv_bfloat16 *__restrict__ dy, int64_t n)
{
    GRID_STRIDE(i, n)
    {
        if (!(bf(y[i]) > 0.f)) dy[i] = tobf(0.f);
    }
}

// db[c] += sum_p dy[p][c]
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ dy, float *__restrict__ db, int64_t npos, int C)
{
    // one block-stride sweep per channel group; C <= 256
    __shared__ float acc[256];
    for (int c = threadIdx.x; c < C; c += blockDim.x) acc[c] = 0.f;
    __syncthreads();
    GRID_STRIDE(i, npos * C) atomicAdd(&acc[i % C], bf(dy[i]));
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], acc[c]);
}

// wt[ci][taps-1-t][co] = w[co][t][ci] (weights of the data-gradient convolution)
__global__ void flip_weights_kernel(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt, int cout,
                                    int taps, int cin)
{
    const int64_t n = (int64_t)cout * taps * cin;
    GRID_STRIDE(i, n)
    {
        const int ci = (int)(i % cin);
        const int t = (int)((i / cin) % taps);
        const int co = (int)(i / ((int64_t)cin * taps));
        wt[((int64_t)ci * taps + (taps - 1 - t)) * cout + co] = w[i];
    }
}

// Adam on FP32 master parameters; refreshes their BF16 copy
// Adam step; lo bounds the parameters from below (-INFINITY: none; 0: projections)
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float lo)
{
    GRID_STRIDE(i, n)
    {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = fmaxf(lo, p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps));
        p[i] = pi;
        if (pb) pb[i] = tobf(pi);
    }
}

// x[z][v][u][0..15]: channel 0 = scale * proj[(z - pad) mod A][v][u] (circular in angle), others 0
__global__ void prepare_input_kernel(const float *__restrict__ proj, __nv_bfloat16 *__restrict__ x, int A, int V,
                                     int U, int Dp, float scale)
{
    const int64_t n = (int64_t)Dp * V * U * 16;
    GRID_STRIDE(i, n)
    {
        const int c = (int)(i % 16);
        const int64_t q = i / 16;
        const int u = (int)(q % U), v = (int)((q / U) % V), z = (int)(q / ((int64_t)U * V));
        float val = 0.f;
        if (c == 0) val = scale * proj[((int64_t)(z % A) * V + v) * U + u];
        x[i] = tobf(val);
    }
}

// head (residual): v = in_scale * base[q] + z[q][0] on the first A slices (base = the
// network's input projections); out = out_scale * max(v, 0); loss = mean 0.5 (v -
// target_scale * target)^2; dz[q][0] = (v - target_scale * target) / n, 0 elsewhere.
__global__ void head_mse_kernel(const float *__restrict__ zin, int cz, const float *__restrict__ base, float in_scale,
                                const float *__restrict__ target, float target_scale, float *__restrict__ out,
                                float out_scale, __nv_bfloat16 *__restrict__ dz, int A, int V, int U, int Dp,
                                double *__restrict__ loss, bool dz16)
{
    const int64_t n = (int64_t)Dp * V * U;
    const double inv_n = 1.0 / ((double)A * V * U);
    double acc = 0.0;
    GRID_STRIDE(q, n)
    {
        const int z = (int)(q / ((int64_t)U * V));
        float g = 0.f;
        if (z < A) {
            const float v = fmaf(in_scale, base[q], zin[q * cz]);
            if (out) out[q] = out_scale * fmaxf(v, 0.f);
            if (target) {
                const float r = v - target_scale * target[q];
                acc += 0.5 * (double)r * (double)r;
                g = (float)((double)r * inv_n);
            }
        }
        if (dz) {
            if (cz == 16 && dz16) {
                // the 16-channel row (g, 0, ..., 0) as two 16-byte stores
                uint4 *d = reinterpret_cast<uint4 *>(dz + q * 16);
                d[0] = make_uint4((unsigned)__bfloat16_as_ushort(tobf(g)), 0u, 0u, 0u);
                d[1] = make_uint4(0u, 0u, 0u, 0u);
            } else {
                dz[q * cz] = tobf(g);
                for (int c = 1; c < cz; ++c) dz[q * cz + c] = tobf(0.f);
            }
        }
    }
    if (loss && target) {
        // one atomic per block: warps reduce by shuffles, then warp 0 over the warps
        __shared__ double part[kT / 32];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            acc = threadIdx.x < (int)(blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (threadIdx.x == 0) atomicAdd(loss, acc * inv_n);
        }
    }
}

// y += x (BF16)
__global__ void add_kernel(const __nv_bfloat16 *__restrict__ x, __nv_bfloat16 *__restrict__ y, int64_t n)
{
    GRID_STRIDE(i, n) y[i] = tobf(bf(y[i]) + bf(x[i]));
}

// out = max |x| (FP32; |x| >= 0 orders like its bit pattern); caller zeroes out
__global__ void absmax_kernel(const float *__restrict__ x, int64_t n, float *__restrict__ out)
{
    float m = 0.f;
    GRID_STRIDE(i, n) m = fmaxf(m, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
}

// projected gradient step g <- max(0, g - eta * grad)
__global__ void projected_step_kernel(float *__restrict__ g, const float *__restrict__ grad, float eta, int64_t n)
{
    GRID_STRIDE(i, n) g[i] = fmaxf(0.f, g[i] - eta * grad[i]);
}

}  // namespace

cudaError_t nn_resample(int op, const void *in, void *out, int D, int H, int W, int C, cudaStream_t s)
{
    const __nv_bfloat16 *a = (const __nv_bfloat16 *)in;
    __nv_bfloat16 *b = (__nv_bfloat16 *)out;
    const int64_t fine = (int64_t)D * H * W * C, coarse = fine / 8;
    if (C % 8 == 0 && aligned16(in, out)) {
        const uint4 *a8 = (const uint4 *)in;
        uint4 *b8 = (uint4 *)out;
        const int G = C / 8;
        switch (op) {
        case 0: pool8_kernel<<<grid_n(coarse / 8), kT, 0, s>>>(a8, b8, D, H, W, G, 0.125f); break;
        case 1: spread8_kernel<<<grid_n(fine / 8), kT, 0, s>>>(a8, b8, D, H, W, G, 0.125f); break;
        case 2: spread8_kernel<<<grid_n(fine / 8), kT, 0, s>>>(a8, b8, D, H, W, G, 1.0f); break;
        case 3: pool8_kernel<<<grid_n(coarse / 8), kT, 0, s>>>(a8, b8, D, H, W, G, 1.0f); break;
        default: return cudaErrorInvalidValue;
        }
        count_launches(1);
        return cudaGetLastError();
    }
    switch (op) {
    case 0: avgpool2_kernel<<<grid_n(coarse), kT, 0, s>>>(a, b, D, H, W, C); break;
    case 1: spread2_kernel<<<grid_n(fine), kT, 0, s>>>(a, b, D, H, W, C, 0.125f); break;
    case 2: spread2_kernel<<<grid_n(fine), kT, 0, s>>>(a, b, D, H, W, C, 1.0f); break;
    case 3: sum2_kernel<<<grid_n(coarse), kT, 0, s>>>(a, b, D, H, W, C); break;
    default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_concat(const void *a, int ca, const void *b, int cb, void *out, int64_t npos, int backward,
                      cudaStream_t s)
{
    if (ca % 8 == 0 && cb % 8 == 0 && aligned16(a, b) && aligned16(out, out)) {
        concat8_kernel<<<grid_n(npos * (ca + cb) / 8), kT, 0, s>>>((const uint4 *)a, ca / 8, (const uint4 *)b, cb / 8,
                                                                   (uint4 *)out, npos, backward);
        count_launches(1);
        return cudaGetLastError();
    }
    if (!backward)
        concat_kernel<<<grid_n(npos * (ca + cb)), kT, 0, s>>>((const __nv_bfloat16 *)a, ca, (const __nv_bfloat16 *)b,
                                                              cb, (__nv_bfloat16 *)out, npos);
    else
        split_kernel<<<grid_n(npos * (ca + cb)), kT, 0, s>>>((const __nv_bfloat16 *)out, (__nv_bfloat16 *)a, ca,
                                                             (__nv_bfloat16 *)b, cb, npos);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_relu_bwd(const void *y, void *dy, int64_t n, cudaStream_t s)
{
    if (n % 8 == 0 && aligned16(y, dy))
        relu_bwd8_kernel<<<grid_n(n / 8), kT, 0, s>>>((const uint4 *)y, (uint4 *)dy, n / 8);
    else
        relu_bwd_kernel<<<grid_n(n), kT, 0, s>>>((const __nv_bfloat16 *)y, (__nv_bfloat16 *)dy, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_bias_grad(const void *dy, float *db, int64_t npos, int C, cudaStream_t s)
{
    if (C % 8 == 0 && kT % (C / 8) == 0 && aligned16(dy, dy))
        bias_grad8_kernel<<<std::min(grid_n(npos * C / 8), 152u * 4u), kT, 0, s>>>((const uint4 *)dy, db, npos, C / 8);
    else
        bias_grad_kernel<<<grid_n(npos * C), kT, 0, s>>>((const __nv_bfloat16 *)dy, db, npos, C);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_flip_weights(const void *w, void *wt, int cout, int taps, int cin, cudaStream_t s)
{
    flip_weights_kernel<<<grid_n((int64_t)cout * taps * cin), kT, 0, s>>>((const __nv_bfloat16 *)w,
                                                                          (__nv_bfloat16 *)wt, cout, taps, cin);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_adam(float *p, const float *g, float *m, float *v, void *pb, int64_t n, float lr, float b1, float b2,
                    float eps, int step, bool nonneg, cudaStream_t s)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<grid_n(n), kT, 0, s>>>(p, g, m, v, (__nv_bfloat16 *)pb, n, lr, b1, b2, eps, c1, c2,
                                         nonneg ? 0.f : -INFINITY);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_prepare_input(const float *proj, void *x, int A, int V, int U, int Dp, float scale, cudaStream_t s)
{
    prepare_input_kernel<<<grid_n((int64_t)Dp * V * U * 16), kT, 0, s>>>(proj, (__nv_bfloat16 *)x, A, V, U, Dp, scale);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_head_mse(const float *z, int cz, const float *base, float in_scale, const float *target,
                        float target_scale, float *out, float out_scale, void *dz, int A, int V, int U, int Dp,
                        double *loss, cudaStream_t s)
{
    if (loss) {
        cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    // few blocks: each ends in one same-address FP64 atomic on the loss
    const bool dz16 = dz && ((uintptr_t)dz & 15) == 0;
    head_mse_kernel<<<std::min(grid_n((int64_t)Dp * V * U), 152u * 4u), kT, 0, s>>>(
        z, cz, base, in_scale, target, target_scale, out, out_scale, (__nv_bfloat16 *)dz, A, V, U, Dp, loss, dz16);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_add(const void *x, void *y, int64_t n, cudaStream_t s)
{
    add_kernel<<<grid_n(n), kT, 0, s>>>((const __nv_bfloat16 *)x, (__nv_bfloat16 *)y, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_absmax(const float *x, int64_t n, float *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    absmax_kernel<<<grid_n(n), kT, 0, s>>>(x, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_projected_step(float *g, const float *grad, float eta, int64_t n, cudaStream_t s)
{
    projected_step_kernel<<<grid_n(n), kT, 0, s>>>(g, grad, eta, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
