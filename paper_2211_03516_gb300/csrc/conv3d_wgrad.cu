// Weight gradient of the 3x3x3 (or 1x1x1) convolution on the 5th-generation tensor cores:
//
//   dW[co][t][ci] += sum_p dY[p][co] X[p + off(t)][ci]      (zero outside the volume)
//
// GEMM mapping: C[m][n] = sum_k A[m][k] B[n][k] with m = t Cin + ci (A = X^T with the taps
// stacked, in M tiles of 128 rows), n = co (B = dY^T, N = Cout), k = output positions.
// A block owns a group of consecutive M tiles (their FP32 accumulators side by side in
// TMEM, Cout columns each) and a range of positions, walked in stages of 32.  Per stage:
//   1. cp.async copies raw channels-last rows into shared memory: for every (dz, dy) that
//      the group's taps use, the 34 positions p0 + dz H W + dy W - 1 ... p0 + dz H W + dy W
//      + 32 (all Cin channels, zeros beyond the array), and the stage's 32 rows of dY.
//      Two raw buffers: the copies for stage c + 1 fly while stage c is transposed.
//   2. every warp transposes 8-channel x 32-position strips into the canonical no-swizzle
//      K-major layout (8-row x 16-byte core matrices, K groups 128 B apart, row groups
//      512 B apart) with ldmatrix.trans + stmatrix.  Lane l supplies the row address of
//      position p0 + l, so the dx shift is an address offset, and a position whose
//      neighbour lies outside the volume (including the wrap across a row end) points
//      at a zero row.
//   3. one issuing thread per tile (lane 0 of warp w issues tiles w, w + nis, ...) issues
//      the stage's two K = 16 MMAs into its tile's accumulator and commits them to the
//      stage's mbarrier, which frees that canonical buffer for stage c + 2.
// At the end each warp reads its TMEM lane quarter and adds the block's partial sums into
// dW with FP32 atomics (consecutive lanes = consecutive rows t Cin + ci of dW: coalesced).
// Every wait is bounded (2 s): on timeout the block sets the error flag, waits (bounded)
// for its own MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace vamrt {
namespace {

using namespace tc;

constexpr int kWThreads = 256;             // 8 warps
constexpr int kKS = 32;                    // positions per stage (= lanes)
constexpr int kRawRows = kKS + 2;          // positions per raw (dz, dy) row
constexpr int kTileBytes = 128 * kKS * 2;  // one M tile of A per stage: 8 KB
constexpr int kRowGroupBytes = kKS * 16;   // 8 rows x 32 positions: 512 B
constexpr int kMaxTpg = 8;
constexpr int kMaxItems = kMaxTpg * 16 + 256 / 8;
constexpr int kBatch = 8;                  // strips a warp transposes per batch

struct WgradArgs {
    const __nv_bfloat16 *X, *dY;
    float *dW;
    int *err;
    int D, H, W, Cin, Cout, taps;
    int Mtot, nmt, tpg;        // A rows (taps x Cin), M tiles, tiles per group
    long long P;               // positions
    int nstage, spb;           // stages of 32 positions in all, per block
    int pairs;                 // (dz, dy) rows per raw X buffer
    int xstride, ystride;      // raw row strides in bytes: 2 Cin + 16, 2 Cout + 16
    int ncols;                 // TMEM columns allocated
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// four 8x8 b16 matrices; lane l gives the address of row l % 8 of matrix l / 8.  After
// .trans register j of lane l holds column l / 4, rows 2 (l % 4) and 2 (l % 4) + 1.
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                              uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}
// the inverse placement without transposition: register j of lane l is row l / 4,
// columns 2 (l % 4) and 2 (l % 4) + 1 of matrix j, whose row r goes to lane 8 j + r's address
__device__ __forceinline__ void stsm_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3)
{
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(r0), "r"(r1),
                 "r"(r2), "r"(r3)
                 : "memory");
}

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

__global__ void __launch_bounds__(kWThreads, 2) conv3d_wgrad_kernel(const WgradArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ uint32_t s_tmem;
    __shared__ int4 items[kMaxItems];
    __shared__ __align__(16) uint4 zero16;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // group of M tiles
    const int g = blockIdx.x;
    const int tile0 = g * a.tpg;
    const int ntile = min(a.tpg, a.nmt - tile0);
    const int row0 = tile0 * 128;
    const int row_end = min(a.Mtot, row0 + ntile * 128);
    const int nis = min(ntile, 8);               // issuing warps
    int t_first = row0 / a.Cin, t_last = (row_end - 1) / a.Cin;
    int dzf, dyf, dxf, dzl, dyl, dxl;
    tap_offset(a.taps, t_first, dzf, dyf, dxf);
    tap_offset(a.taps, t_last, dzl, dyl, dxl);
    const int pair_first = (dzf + 1) * 3 + (dyf + 1);
    const int npairs = (dzl + 1) * 3 + (dyl + 1) - pair_first + 1;
    const long long HW = (long long)a.H * a.W;

    // shared-memory carve-up (dynamic part 1024-aligned)
    unsigned char *base = smem_raw;
    const uint32_t canonA = smem_u32(base);
    const uint32_t canonA_bytes = (uint32_t)a.tpg * kTileBytes;
    const uint32_t canonB = canonA + 2 * canonA_bytes;
    const uint32_t canonB_bytes = (uint32_t)a.Cout / 8 * kRowGroupBytes;
    const uint32_t rawX = canonB + 2 * canonB_bytes;
    const uint32_t rawX_bytes = (uint32_t)a.pairs * kRawRows * a.xstride;
    const uint32_t rawY = rawX + 2 * rawX_bytes;
    const uint32_t rawY_bytes = (uint32_t)kKS * a.ystride;
    const uint32_t zero_addr = smem_u32(&zero16);

    // work items: A row groups (8 rows = 8 channels of one tap) then B row groups
    const int nA = (row_end - row0) / 8, nB = a.Cout / 8, nitems = nA + nB;
    for (int it = tid; it < nitems; it += kWThreads) {
        int4 e;
        if (it < nA) {
            const int r = row0 + it * 8;
            const int t = r / a.Cin, ci0 = r - t * a.Cin;
            int dz, dy, dx;
            tap_offset(a.taps, t, dz, dy, dx);
            const int slot = (dz + 1) * 3 + (dy + 1) - pair_first;
            e.x = slot * kRawRows * a.xstride + (dx + 1) * a.xstride + ci0 * 2;
            e.y = it * kRowGroupBytes;                        // tile (it / 16) x 8 KB + (it % 16) x 512
            e.z = (dz + 1) | (dy + 1) << 2 | (dx + 1) << 4;
        } else {
            const int cg = it - nA;
            e.x = cg * 16;
            e.y = cg * kRowGroupBytes;
            e.z = 256;
        }
        e.w = 0;
        items[it] = e;
    }
    if (tid == 0) {
        zero16 = make_uint4(0, 0, 0, 0);
        mbar_init(smem_u32(&bars[0]), nis);
        mbar_init(smem_u32(&bars[1]), nis);
        mbar_init_fence();
    }
    if (warp == 0) tmem_alloc(smem_u32(&s_tmem), a.ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    const int s_begin = blockIdx.y * a.spb;
    const int n = max(0, min(a.spb, a.nstage - s_begin));
    const uint32_t idesc = instr_desc(128, a.Cout);

    // raw-row copies of stage st into buffer b (issued by every thread, one commit group)
    const int cpr = a.Cin / 8, cpy = a.Cout / 8;
    const int xr0 = tid / cpr, xh = tid - xr0 * cpr, xstep = kWThreads / cpr;
    const int yr0 = tid / cpy, yh = tid - yr0 * cpy, ystep = kWThreads / cpy;
    auto load_raw = [&](int st, int b) {
        const long long p0 = (long long)st * kKS;
        if (xr0 < xstep) {
            for (int r = xr0; r < npairs * kRawRows; r += xstep) {
                const int j = r / kRawRows, q = r - j * kRawRows;
                const int pair = pair_first + j;
                const long long src = p0 + (long long)(pair / 3 - 1) * HW + (long long)(pair % 3 - 1) * a.W - 1 + q;
                const bool ok = src >= 0 && src < a.P;
                cp_async16_zfill(rawX + b * rawX_bytes + (uint32_t)(j * kRawRows + q) * a.xstride + xh * 16,
                                 ok ? (const void *)(a.X + src * a.Cin + xh * 8) : (const void *)a.X, ok ? 16 : 0);
            }
        }
        if (yr0 < ystep) {
            for (int q = yr0; q < kKS; q += ystep) {
                const long long src = p0 + q;
                const bool ok = src < a.P;
                cp_async16_zfill(rawY + b * rawY_bytes + (uint32_t)q * a.ystride + yh * 16,
                                 ok ? (const void *)(a.dY + src * a.Cout + yh * 8) : (const void *)a.dY,
                                 ok ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    // this lane's position p0 + lane as (z, y, x), advanced by 32 per stage
    long long p = (long long)s_begin * kKS + lane;
    int z = (int)(p / HW);
    int y = (int)((p - (long long)z * HW) / a.W);
    int x = (int)(p - (long long)z * HW - (long long)y * a.W);

    bool ok = true;
    int c_done = -1;                                  // last stage whose MMAs were issued
    if (n > 0) load_raw(s_begin, 0);
    for (int c = 0; c < n; ++c) {
        const int buf = c & 1;
        if (c + 1 < n) load_raw(s_begin + c + 1, buf ^ 1);
        else cp_async_commit();
        cp_async_wait_1();
        bool mine = true;
        if (c >= 2) mine = mbar_wait(smem_u32(&bars[buf]), ((c - 2) >> 1) & 1);
        if (!__syncthreads_and(mine)) { ok = false; break; }

        // neighbour validity of this lane's position: bit d + 1 for offset d
        const unsigned zok = ((unsigned)(z - 1) < (unsigned)a.D) | ((unsigned)z < (unsigned)a.D) << 1 |
                             ((unsigned)(z + 1) < (unsigned)a.D) << 2;
        const unsigned yok = ((unsigned)(y - 1) < (unsigned)a.H) | ((unsigned)y < (unsigned)a.H) << 1 |
                             ((unsigned)(y + 1) < (unsigned)a.H) << 2;
        const unsigned xok = ((unsigned)(x - 1) < (unsigned)a.W) | ((unsigned)x < (unsigned)a.W) << 1 |
                             ((unsigned)(x + 1) < (unsigned)a.W) << 2;
        const uint32_t rx = rawX + buf * rawX_bytes + lane * a.xstride;
        const uint32_t ry = rawY + buf * rawY_bytes + lane * a.ystride;
        const uint32_t ca = canonA + buf * canonA_bytes + lane * 16;
        const uint32_t cb = canonB + buf * canonB_bytes + lane * 16;
        // kBatch items per warp at a time: every load issued before the first store
        for (int it0 = warp; it0 < nitems; it0 += kBatch * (kWThreads / 32)) {
            uint32_t r[kBatch][4], dst[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int it = it0 + u * (kWThreads / 32);
                if (it < nitems) {
                    const int4 e = items[it];
                    uint32_t src;
                    if (e.z & 256) {
                        src = ry + e.x;
                        dst[u] = cb + e.y;
                    } else {
                        const unsigned v =
                            (zok >> (e.z & 3)) & (yok >> ((e.z >> 2) & 3)) & (xok >> ((e.z >> 4) & 3)) & 1u;
                        src = v ? rx + e.x : zero_addr;
                        dst[u] = ca + e.y;
                    }
                    ldsm_x4_trans(src, r[u][0], r[u][1], r[u][2], r[u][3]);
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                if (it0 + u * (kWThreads / 32) < nitems) stsm_x4(dst[u], r[u][0], r[u][1], r[u][2], r[u][3]);
        }
        fence_proxy_async();
        __syncthreads();
        if (lane == 0 && warp < nis) {
            tc_fence_after();
            const uint32_t a0 = canonA + buf * canonA_bytes, b0 = canonB + buf * canonB_bytes;
            for (int i = warp; i < ntile; i += nis) {
#pragma unroll
                for (int s = 0; s < 2; ++s)
                    mma_bf16(tmem + (uint32_t)(i * a.Cout), smem_desc(a0 + i * kTileBytes + s * 256, 128, 512),
                             smem_desc(b0 + s * 256, 128, 512), idesc, (c > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&bars[buf]));
        }
        c_done = c;
        x += kKS;
        while (x >= a.W) {
            x -= a.W;
            if (++y == a.H) { y = 0; ++z; }
        }
    }
    cp_async_wait_all();
    if (ok && c_done >= 0) {
        const bool mine = mbar_wait(smem_u32(&bars[c_done & 1]), (c_done >> 1) & 1);
        ok = __syncthreads_and(mine);
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            if (c_done >= 0) (void)mbar_wait(smem_u32(&bars[c_done & 1]), (c_done >> 1) & 1);
        }
    } else if (c_done >= 0) {
        tc_fence_after();
        const int q = warp & 3;
        for (int i = warp >> 2; i < ntile; i += 2) {
            const int R = row0 + i * 128 + q * 32 + lane;
            for (int co0 = 0; co0 < a.Cout; co0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(i * a.Cout + co0), v);
                if (R < row_end) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(a.dW + (long long)(co0 + j) * a.Mtot + R, v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.ncols);
}

// number of (dz, dy) rows the taps of rows [r0, r1) use
int pairs_of(int taps, int Cin, int r0, int r1)
{
    if (taps == 1) return 1;
    const int tf = r0 / Cin, tl = (r1 - 1) / Cin;
    return tl / 3 - tf / 3 + 1;
}

}  // namespace

cudaError_t launch_conv3d_wgrad_tc(const void *X, const void *dY, float *dW, int D, int H, int W, int Cin, int Cout,
                                   int taps, int *err, cudaStream_t s)
{
    WgradArgs a{};
    a.X = (const __nv_bfloat16 *)X;
    a.dY = (const __nv_bfloat16 *)dY;
    a.dW = dW;
    a.err = err;
    a.D = D; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout; a.taps = taps;
    a.Mtot = taps * Cin;
    a.nmt = (a.Mtot + 127) / 128;
    a.P = (long long)D * H * W;
    a.nstage = (int)((a.P + kKS - 1) / kKS);
    a.xstride = 2 * Cin + 16;
    a.ystride = 2 * Cout + 16;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;

    // tiles per group: two blocks per SM if their shared memory and TMEM columns allow it,
    // else one; groups balanced in size
    int per_sm = 0;
    size_t smem = 0;
    for (int bps = 2; bps >= 1 && !per_sm; --bps) {
        const size_t budget = bps == 2 ? 108 * 1024 : 220 * 1024;   // beside ~3 KB static + 1 KB reserved
        const int colcap = 512 / bps;
        for (int tpg = std::min(kMaxTpg, std::min(a.nmt, colcap / Cout)); tpg >= 1; --tpg) {
            const int ng = (a.nmt + tpg - 1) / tpg;
            const int t2 = (a.nmt + ng - 1) / ng;
            int pairs = 0;
            for (int gi = 0; gi * t2 < a.nmt; ++gi)
                pairs = std::max(pairs, pairs_of(taps, Cin, gi * t2 * 128, std::min(a.Mtot, (gi + 1) * t2 * 128)));
            const size_t need = 2 * ((size_t)t2 * kTileBytes + (size_t)Cout / 8 * kRowGroupBytes +
                                     (size_t)pairs * kRawRows * a.xstride + (size_t)kKS * a.ystride);
            if (need <= budget) {
                a.tpg = t2;
                a.pairs = pairs;
                smem = need;
                per_sm = bps;
                break;
            }
        }
    }
    if (!per_sm) return cudaErrorNotSupported;
    const int ngroups = (a.nmt + a.tpg - 1) / a.tpg;
    int ncols = 32;
    while (ncols < a.tpg * Cout) ncols <<= 1;
    a.ncols = ncols;
    // at most one wave: a block more than the resident slots would double the time
    const int target = per_sm * sms;
    int nsplit = std::max(1, target / ngroups);
    a.spb = (a.nstage + nsplit - 1) / nsplit;
    nsplit = (a.nstage + a.spb - 1) / a.spb;
    cudaError_t e = cudaFuncSetAttribute(conv3d_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conv3d_wgrad_kernel<<<dim3(ngroups, nsplit), kWThreads, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
