// Weight gradient of the 3x3x3 (or 1x1x1) convolution on the 5th-generation tensor cores:
//
//   dW[co][t][ci] += sum_p dY[p][co] X[p + off(t)][ci]      (zero outside the volume)
//
// GEMM mapping: C[m][n] = sum_k A[m][k] B[n][k] with m = t Cin + ci (A = X^T with the taps
// stacked, in M tiles of 128 rows), n = co (B = dY^T, N = Cout), k = output positions.  A
// block owns a group of consecutive M tiles (FP32 accumulators side by side in TMEM) and
// a range of positions walked in stages of KS; at the end it adds its partial sums into
// dW with FP32 atomics (consecutive lanes = consecutive rows t Cin + ci: coalesced).
// Every wait is bounded (2 s): on timeout the block sets the error flag, waits (bounded)
// for its own MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace vamrt {
namespace {

using namespace tc;

constexpr int kMaxTpg = 8;

// tap t -> (dz, dy, dx) in -1..1 (taps == 1: the centre)
__device__ __forceinline__ void tap_offset(int taps, int t, int &dz, int &dy, int &dx)
{
    if (taps == 27) {
        dz = t / 9 - 1;
        dy = (t / 3) % 3 - 1;
        dx = t % 3 - 1;
    } else {
        dz = dy = dx = 0;
    }
}

// ---------------------------------------------------------------------------------
// TMA-fed kernel: no transposition.  The tensor cores also take operands MN-major (M or N
// contiguous).  For A = X^T (M = t Cin + ci, K = positions) a column block of cw rows
// (tap t, channels c0 .. c0 + cw - 1) over a stage's KS positions is X[p + off(t)][c0 ..
// c0 + cw - 1], p = p0 .. p0 + KS - 1: KS rows of 2 cw bytes -- exactly what a TMA tile
// load of box {cw channels, BX x, 1 y, 1 z} at (c0, x + dx, y + dy, z + dz) writes, with
// the zero fill of out-of-range coordinates supplying the convolution's zero padding
// (including x = -1 and x = W).  cw = 16, 32 or 64 channels (the widest dividing Cin), so
// rows are 32, 64 or 128 bytes in the matching TMA swizzle, which is the tensor cores'
// swizzled MN-major layout: column blocks LBO = KS x 2 cw bytes apart, 8-row K groups
// SBO = 16 cw bytes apart.  B = dY^T likewise, blocks of cwB output channels, boxes
// {cwB, KS} of dY viewed as [P][Cout].
// Block: warp 0 issues the stage's boxes (lane 0 arms the stage's mbarrier with the byte
// count), lane 0 of warps 4-7 issues the MMAs (accumulator = one M tile x K-step part, kp
// parts per tile so that small groups still keep several issuers), all warps run the
// epilogue.  A ring of stage slots, full/empty mbarriers per slot, bounded waits.
// ---------------------------------------------------------------------------------
constexpr int kTThreads = 256;
constexpr int kTIssuer0 = 4, kTIssuers = 4;
constexpr int kTMaxSlots = 4;

struct TmaArgs {
    float *dW;
    int *err;
    int D, H, W, Cin, Cout, taps;
    int Mtot, nmt, tpg, kp;    // A rows, M tiles, tiles per group, accumulators per tile
    int KS, BX;                // positions per stage and per X box (BX divides W and KS)
    int nstage, spb;           // stages in all, per block
    int slots, slot_bytes;     // ring of stage slots: B blocks, then the group's A blocks
    int cwA, cwB;              // channels per column block (16, 32 or 64: 32/64/128-byte rows)
    int ncols;
};

// UMMA layout type of a swizzled MN-major operand whose rows are cw x 2 bytes
__host__ __device__ __forceinline__ uint32_t swizzle_layout(int cw) { return cw == 64 ? 2u : cw == 32 ? 4u : 6u; }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(kTThreads, 2)
    conv3d_wgrad_tma_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
                            const TmaArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2 * kTMaxSlots + 1];   // full[slots], empty[slots], done
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_fin;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile0 = blockIdx.x * a.tpg;
    const int ntile = min(a.tpg, a.nmt - tile0);
    const int row0 = tile0 * 128, row_end = min(a.Mtot, row0 + ntile * 128);
    const int nAb = (row_end - row0) / a.cwA, nBb = a.Cout / a.cwB;     // column blocks loaded
    const int nacc = ntile * a.kp, nis = min(kTIssuers, nacc);
    const int rowA = 2 * a.cwA, rowB = 2 * a.cwB;                          // bytes per K row
    const int blkA = a.KS * rowA, blkB = a.KS * rowB;
    const int Bbytes = nBb * blkB;
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kTMaxSlots]);
    const uint32_t done = smem_u32(&bars[2 * kTMaxSlots]);

    if (tid == 0) {
        for (int s = 0; s < a.slots; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, nis);
        }
        mbar_init(done, nis);
        mbar_init_fence();
        s_abort = 0;
        s_fin = 0;
    }
    if (warp == kTIssuer0) tmem_alloc(smem_u32(&s_tmem), a.ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int s_begin = blockIdx.y * a.spb;
    const int n = max(0, min(a.spb, a.nstage - s_begin));

    if (warp == 0) {
        // ---- producer: the stage's A boxes (plane it, box b) and B planes, spread over the lanes ----
        const long long HW = (long long)a.H * a.W;
        const int nbx = a.KS / a.BX;
        const uint32_t tx = (uint32_t)(nAb * blkA + Bbytes);
        for (int c = 0; c < n; ++c) {
            const int slot = c % a.slots;
            bool ok = true;
            if (c >= a.slots) ok = mbar_wait(empty0 + 8 * slot, (c / a.slots - 1) & 1);
            if (!__all_sync(0xffffffffu, ok) || __any_sync(0xffffffffu, s_abort)) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicExch(a.err, 1);
                }
                break;
            }
            const uint32_t sb = base + slot * a.slot_bytes, bar = full0 + 8 * slot;
            if (lane == 0) mbar_arrive_expect_tx(bar, tx);
            __syncwarp();
            const long long p0 = (long long)(s_begin + c) * a.KS;
            for (int k = lane; k < nAb * nbx + nBb; k += 32) {
                if (k < nBb) {
                    tma_load_2d(sb + k * blkB, &ymap, a.cwB * k, (int)p0, bar);
                } else {
                    const int j = (k - nBb) / nbx, b = k - nBb - j * nbx;
                    const int r = row0 + j * a.cwA, t = r / a.Cin, c0 = r - t * a.Cin;
                    int dz, dy, dx;
                    tap_offset(a.taps, t, dz, dy, dx);
                    const long long p = p0 + (long long)b * a.BX;
                    const int z = (int)(p / HW);
                    const long long rem = p - (long long)z * HW;
                    const int y = (int)(rem / a.W), x = (int)(rem - (long long)y * a.W);
                    tma_load_4d(sb + Bbytes + j * blkA + b * a.BX * rowA, &xmap, c0, x + dx, y + dy, z + dz, bar);
                }
            }
        }
    } else if (warp >= kTIssuer0 && warp - kTIssuer0 < nis) {
        // ---- issuers: accumulators k0, k0 + nis, ... = (tile acc / kp, K-step part acc % kp) ----
        if (lane == 0) {
            const int k0 = warp - kTIssuer0, nks = a.KS / 16;
            const uint32_t idesc = instr_desc(128, a.Cout) | (1u << 15) | (1u << 16);   // A, B MN-major
            const uint64_t swA = (uint64_t)swizzle_layout(a.cwA) << 61, swB = (uint64_t)swizzle_layout(a.cwB) << 61;
            for (int c = 0; c < n; ++c) {
                const int slot = c % a.slots;
                if (!mbar_wait(full0 + 8 * slot, (c / a.slots) & 1) || s_abort) {
                    s_abort = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t sb = base + slot * a.slot_bytes;
                for (int acc = k0; acc < nacc; acc += nis) {
                    const int i = acc / a.kp, part = acc - i * a.kp;
                    for (int s = part; s < nks; s += a.kp)
                        mma_bf16(tmem + (uint32_t)(acc * a.Cout),
                                 smem_desc(sb + Bbytes + i * (128 / a.cwA) * blkA + s * 16 * rowA, blkA, 8 * rowA) | swA,
                                 smem_desc(sb + s * 16 * rowB, blkB, 8 * rowB) | swB, idesc,
                                 (c > 0 || s != part) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * slot);
            }
            mma_commit(done);
        }
        __syncwarp();
    }
    __syncthreads();
    if (tid == 0) {
        s_fin = mbar_wait(done, 0) ? 1 : 0;     // every MMA issued has completed
        if (!s_fin) atomicExch(a.err, 1);
    }
    __syncthreads();
    tc_fence_after();
    if (s_fin && !s_abort && n > 0) {
        const int q = warp & 3;
        for (int i = warp >> 2; i < ntile; i += kTThreads / 128) {
            const int R = row0 + i * 128 + q * 32 + lane;
            for (int co0 = 0; co0 < a.Cout; co0 += 16) {
                float sum[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(i * a.kp * a.Cout + co0), sum);
                for (int part = 1; part < a.kp; ++part) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((i * a.kp + part) * a.Cout + co0), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[j] += v[j];
                }
                if (R < row_end) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(a.dW + (long long)(co0 + j) * a.Mtot + R, sum[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kTIssuer0) tmem_dealloc(tmem, a.ncols);
}

int sm_count_wgrad()
{
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 148;
    return sms;
}

// TMA-fed kernel: stages of 64 positions where W allows (else 32), the largest tile group
// whose ring of three slots and accumulators fit two blocks per SM (else one); returns
// cudaErrorNotSupported for what it cannot take
cudaError_t launch_wgrad_tma(const void *X, const void *dY, float *dW, int D, int H, int W, int Cin, int Cout,
                             int taps, int *err, cudaStream_t s)
{
    const long long P = (long long)D * H * W;
    if (((uintptr_t)X & 15) || ((uintptr_t)dY & 15) || P >= (1ll << 31)) return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc) return cudaErrorNotSupported;
    WgradPlan pl;
    if (!plan_wgrad_tma(D, H, W, Cin, Cout, taps, sm_count_wgrad(), &pl)) return cudaErrorNotSupported;
    TmaArgs a{};
    a.dW = dW;
    a.err = err;
    a.D = D; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout; a.taps = taps;
    a.Mtot = pl.Mtot; a.nmt = pl.nmt; a.tpg = pl.tpg; a.kp = pl.kp;
    a.KS = pl.KS; a.BX = pl.BX; a.nstage = pl.nstage; a.spb = pl.spb;
    a.slots = pl.slots; a.slot_bytes = pl.slot_bytes; a.cwA = pl.cwA; a.cwB = pl.cwB; a.ncols = pl.ncols;

    CUtensorMap xmap, ymap;
    const cuuint64_t xdims[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
    const cuuint64_t xstr[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t xbox[4] = {(cuuint32_t)a.cwA, (cuuint32_t)a.BX, 1, 1};
    const cuuint64_t ydims[2] = {(cuuint64_t)Cout, (cuuint64_t)P};
    const cuuint64_t ystr[1] = {(cuuint64_t)Cout * 2};
    const cuuint32_t ybox[2] = {(cuuint32_t)a.cwB, (cuuint32_t)a.KS};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    auto swz = [](int cw) {
        return cw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : cw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
    };
    if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(X), xdims, xstr, xbox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz(a.cwA), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(dY), ydims, ystr, ybox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz(a.cwB), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;

    const size_t smem = (size_t)a.slots * a.slot_bytes;
    cudaError_t e = cudaFuncSetAttribute(conv3d_wgrad_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv3d_wgrad_tma_kernel<<<dim3(pl.ngroups, pl.nsplit), kTThreads, smem, s>>>(xmap, ymap, a);
    return cudaGetLastError();
}

}  // namespace

// Plan of the TMA-fed weight gradient: stages of 64 positions where W allows (else 32;
// boxes of BX positions, BX dividing W and KS), column blocks of cwA / cwB channels (the
// widest of 64, 32, 16 dividing Cin / Cout), the largest tile group whose ring of three
// or four slots and accumulators fit two blocks per SM (else one), groups balanced in
// size, and the positions split so that the grid is at most one wave.
bool plan_wgrad_tma(int D, int H, int W, int Cin, int Cout, int taps, int sms, WgradPlan *pl)
{
    if (W < 16 || W % 16 || Cin % 16 || Cout % 16 || Cout > 256 || sms < 1 || (taps != 1 && taps != 27))
        return false;
    const long long P = (long long)D * H * W;
    if (P < 1 || P >= (1ll << 31)) return false;
    WgradPlan a{};
    a.Mtot = taps * Cin;
    a.nmt = (a.Mtot + 127) / 128;
    a.KS = W % 64 == 0 ? 64 : 32;
    a.BX = W % a.KS == 0 ? a.KS : 16;
    a.nstage = (int)((P + a.KS - 1) / a.KS);
    a.cwA = Cin % 64 == 0 ? 64 : Cin % 32 == 0 ? 32 : 16;
    a.cwB = Cout % 64 == 0 ? 64 : Cout % 32 == 0 ? 32 : 16;
    for (int bps = 2; bps >= 1 && !a.per_sm; --bps) {
        const int budget = bps == 2 ? 108 * 1024 : 220 * 1024;
        for (int tpg = std::min(kMaxTpg, std::min(a.nmt, (512 / bps) / Cout)); tpg >= 1; --tpg) {
            const int ng = (a.nmt + tpg - 1) / tpg;
            const int t2 = (a.nmt + ng - 1) / ng;
            const int slot = ((Cout + 128 * t2) * a.KS * 2 + 1023) / 1024 * 1024;
            const int slots = std::min(kTMaxSlots, budget / slot);
            if (slots < 3) continue;
            int kp = std::min(a.KS / 16, std::max(1, kTIssuers / t2));
            while (kp > 1 && t2 * kp * Cout > 512 / bps) --kp;
            a.tpg = t2;
            a.kp = kp;
            a.slots = slots;
            a.slot_bytes = slot;
            a.per_sm = bps;
            break;
        }
    }
    if (!a.per_sm) return false;
    a.ncols = 32;
    while (a.ncols < a.tpg * a.kp * Cout) a.ncols <<= 1;
    a.ngroups = (a.nmt + a.tpg - 1) / a.tpg;
    a.nsplit = std::max(1, a.per_sm * sms / a.ngroups);      // at most one wave
    a.spb = (a.nstage + a.nsplit - 1) / a.nsplit;
    a.nsplit = (a.nstage + a.spb - 1) / a.spb;
    *pl = a;
    return true;
}

PFN_cuTensorMapEncodeTiled_v12000 tma_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

cudaError_t launch_conv3d_wgrad_tc(const void *X, const void *dY, float *dW, int D, int H, int W, int Cin, int Cout,
                                   int taps, int *err, cudaStream_t s)
{
    const cudaError_t e = launch_wgrad_tma(X, dY, dW, D, H, W, Cin, Cout, taps, err, s);
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace vamrt
