// 3x3x3 (or 1x1x1) convolution, stride 1, zero padding, as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05): BF16 operands staged in shared memory, FP32
// accumulator in tensor memory (TMEM), one elected thread issuing the MMAs.
//
//   Y[p][co] = act( bias[co] + sum_{t, ci} X[p + off(t)][ci] * Wt[co][t][ci] )
//
// Layouts (all channels-last): X [D][H][W][Cin] bf16, Cin a multiple of 16;
// Wt [Cout][taps][Cin] bf16 (GEMM rows of K = taps * Cin, K-major); Y [D][H][W][Cout]
// bf16 or fp32, Cout a multiple of 16 (<= 256).  Out-of-volume taps read zeros.
//
// GEMM mapping: M = 128 consecutive output positions (TMEM lanes), N = Cout (TMEM
// columns), K in chunks of 16 channels of one tap.  A block of 128 threads: thread i
// gathers row i of every A chunk (32 bytes: 16 channels of one neighbour) and part of
// the B chunk into the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices; 128 B between K groups, 256 B between row groups).  Two stages: while the
// tensor core runs chunk c, the threads stage chunk c+1; an mbarrier signalled by
// tcgen05.commit releases each stage.  Every wait is bounded: on timeout the block sets
// the error flag, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace vamrt {
namespace {

constexpr int kConvThreads = 128;      // 4 warps = the 4 TMEM lane quarters
constexpr int kM = 128;
constexpr int kStageA = kM * 16 * 2;   // 4 KB
constexpr int kMaxCout = 256;
constexpr int kStageB = kMaxCout * 16 * 2;   // 8 KB
using namespace tc;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) { return tc::smem_desc(addr, 128, 256); }
__device__ __forceinline__ uint32_t instr_desc(int n) { return tc::instr_desc(kM, n); }

// byte offset of element row r, 16-byte half h (channels 8h..8h+7) in a staged tile
__device__ __forceinline__ int core_off(int r, int h) { return (r >> 3) * 256 + h * 128 + (r & 7) * 16; }

template <int TAPS, typename OT>
__global__ void __launch_bounds__(kConvThreads)
    conv3d_tc_kernel(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ Wt,
                     const float *__restrict__ bias, OT *__restrict__ Y, int D, int H, int W, int Cin, int Cout,
                     int relu, int *__restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                       // 2 stages of A
    unsigned char *sB = smem + 2 * kStageA;         // 2 stages of B
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t P = (int64_t)D * H * W;
    const int64_t p0 = (int64_t)blockIdx.x * kM;
    int ncols = 32;
    while (ncols < Cout) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // this thread's output position (row of the A tile)
    const int64_t p = p0 + tid;
    const bool pvalid = p < P;
    int z = 0, y = 0, x = 0;
    if (pvalid) {
        x = (int)(p % W);
        y = (int)((p / W) % H);
        z = (int)(p / ((int64_t)W * H));
    }
    const int cchunks = Cin >> 4;
    const int nchunks = TAPS * cchunks;
    const uint32_t idesc = instr_desc(Cout);
    bool ok = true;

    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (c >= 2) {
            // stage s is free once the MMA of chunk c-2 (its (c-2)/2-th commit) completed
            const bool mine = mbar_wait(smem_u32(&bars[s]), ((c - 2) >> 1) & 1);
            if (!__syncthreads_and(mine)) { ok = false; break; }
        }
        const int t = c / cchunks, cc = c - t * cchunks;
        int dz = 0, dy = 0, dx = 0;
        if (TAPS == 27) { dz = t / 9 - 1; dy = (t / 3) % 3 - 1; dx = t % 3 - 1; }
        // A: row tid = 16 channels of the neighbour at offset (dz, dy, dx)
        uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0;
        const int zz = z + dz, yy = y + dy, xx = x + dx;
        if (pvalid && zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W) {
            const uint4 *src = reinterpret_cast<const uint4 *>(
                X + ((((int64_t)zz * H + yy) * W + xx) * Cin + cc * 16));
            a0 = __ldg(src);
            a1 = __ldg(src + 1);
        }
        unsigned char *A = sA + s * kStageA;
        *reinterpret_cast<uint4 *>(A + core_off(tid, 0)) = a0;
        *reinterpret_cast<uint4 *>(A + core_off(tid, 1)) = a1;
        // B: rows co = tid, tid + 128 (Cout <= 256)
        unsigned char *Bs = sB + s * kStageB;
        for (int co = tid; co < Cout; co += kConvThreads) {
            const uint4 *src = reinterpret_cast<const uint4 *>(Wt + (((int64_t)co * TAPS + t) * Cin + cc * 16));
            *reinterpret_cast<uint4 *>(Bs + core_off(co, 0)) = __ldg(src);
            *reinterpret_cast<uint4 *>(Bs + core_off(co, 1)) = __ldg(src + 1);
        }
        // generic-proxy smem writes -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            mma_bf16(tmem, smem_desc(smem_u32(A)), smem_desc(smem_u32(Bs)), idesc, c > 0 ? 1u : 0u);
            mma_commit(smem_u32(&bars[s]));
        }
    }
    if (ok && nchunks > 0) {
        // the last commit completes once every MMA issued before it has completed
        const int c = nchunks - 1;
        const bool mine = mbar_wait(smem_u32(&bars[c & 1]), (c >> 1) & 1);
        ok = __syncthreads_and(mine);
    }
    if (!ok) {
        // give the MMAs already issued one more bounded chance to drain before TMEM is freed
        if (tid == 0) {
            atomicExch(err, 1);
            for (int s2 = 0; s2 < 2; ++s2) (void)mbar_wait(smem_u32(&bars[s2]), 0);
        }
    } else {
        tc_fence_after();
        // epilogue: lane quarter `warp` of TMEM holds rows 32 warp .. 32 warp + 31
        const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int n0 = 0; n0 < Cout; n0 += 16) {
            float v[16];
            tmem_ld16(row_addr + (uint32_t)n0, v);
            if (pvalid) {
                OT *dst = Y + p * Cout + n0;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float r = v[i] + (bias ? bias[n0 + i] : 0.f);
                    if (relu) r = fmaxf(r, 0.f);
                    if constexpr (sizeof(OT) == 2)
                        dst[i] = __float2bfloat16_rn(r);
                    else
                        dst[i] = r;
                }
            }
        }
        (void)lane;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

cudaError_t launch_conv3d_tc(const void *X, const void *Wt, const float *bias, void *Y, int out_f32, int D, int H,
                             int W, int Cin, int Cout, int taps, int relu, int *err, cudaStream_t s)
{
    // the halo-tile kernel takes every shape with W % 8 == 0; this gather kernel the rest
    cudaError_t e = launch_conv3d_halo(X, Wt, bias, Y, out_f32, D, H, W, Cin, Cout, taps, relu, err, s);
    if (e != cudaErrorNotSupported) return e;
    const int64_t P = (int64_t)D * H * W;
    const unsigned grid = (unsigned)((P + kM - 1) / kM);
    const size_t smem = 2 * kStageA + 2 * kStageB;
    const __nv_bfloat16 *x = (const __nv_bfloat16 *)X, *w = (const __nv_bfloat16 *)Wt;
#define VAMRT_CONV(T, OT)                                                                                         \
    do {                                                                                                          \
        e = cudaFuncSetAttribute(conv3d_tc_kernel<T, OT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e == cudaSuccess)                                                                                     \
            conv3d_tc_kernel<T, OT><<<grid, kConvThreads, smem, s>>>(x, w, bias, (OT *)Y, D, H, W, Cin, Cout, relu, \
                                                                     err);                                        \
    } while (0)
    if (taps == 27) {
        if (out_f32) VAMRT_CONV(27, float); else VAMRT_CONV(27, __nv_bfloat16);
    } else {
        if (out_f32) VAMRT_CONV(1, float); else VAMRT_CONV(1, __nv_bfloat16);
    }
#undef VAMRT_CONV
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
