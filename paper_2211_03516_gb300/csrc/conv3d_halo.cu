// Halo-tiled 3x3x3 (or 1x1x1) convolution on the 5th-generation tensor cores: a
// persistent, warp-specialised implicit GEMM.
//
//   Y[p][co] = act( bias[co] + sum_{t, ci} X[p + off(t)][ci] * Wt[co][t][ci] )
//
// Same operation and layouts as conv3d_tc.cu (X [D][H][W][Cin] bf16, Wt [Cout][taps][Cin],
// Y [D][H][W][Cout] bf16 or fp32, zero padding); this kernel needs W % 8 == 0, W <= 240
// (a row is one TMA box dimension) and a 16-byte aligned X.
//
// Slot layout.  A work item is a region of TZ output planes x TY output rows x all W
// columns (and a slice of Nt output channels).  Its input tile -- (TZ + 2) planes x
// (TY + 2) rows with the one-voxel halo -- is staged one 16-channel chunk at a time as a
// run of 32-byte "slots" (16 bf16 channels of one voxel).  A row takes WP = W + 16 slots,
// x = -8 .. W + 7: voxel x sits in slot x + 8, and the zero slots around it are its x = -1
// and x = W neighbours.
//
// GEMM mapping.  M = 128 consecutive slots of the region (TMEM lanes), K = 16 channels per
// MMA.  Because the slot index is linear in (z, y, x), the A operand of taps (dz, dy, *)
// for a tile is the same slot run shifted by dz PT + dy WP slots: one shared-memory
// descriptor per (tile, dz, dy), no data movement.  The three dx taps share that A and are
// stacked in N (N = 3 Nt: columns dx, then output channel), so row m of the accumulator
// holds, per dx, the (dz, dy)-summed product at slot m; the epilogue forms
// Y[m] = D[m - 1][dx = -1] + D[m][0] + D[m + 1][+1].  A is K-major in the 32-byte swizzle
// (8-slot atoms of 256 bytes, SBO = 256 B); every tile start and shift is a whole atom.
// For W = 128 a tile is one row (its neighbours beyond the tile are pads); otherwise tiles
// run through each plane's rows 120 slots apart with one margin row at either end.  Rows in
// padding or beyond the region are computed and discarded.  B (weights of one chunk, all
// taps) is staged in the canonical K-major no-swizzle layout.
//
// Staging: one TMA tile load per chunk, box {16 channels, WP x from -8, TY + 2 rows, TZ + 2
// planes}, writes the whole input tile in that swizzled layout; its zero fill supplies the
// row pads and the halo outside the volume.  The weights come by cp.async from four loader
// warps.  (Boxes of 16-byte rows -- 8 channels -- and cp.async copies of the tile both moved
// about 24 B/cycle/SM; 32-byte rows roughly double that.)
//
// Roles (544 threads): warps 0-7 drain TMEM in two sets of four, alternate tiles (warp
// 4 s + w owns lanes 32w..32w+31) and write Y; warps 8-11 stage input tiles (TMA) and
// weights (cp.async) into two shared-memory stages; lane 0 of each of warps 12-16 issues
// the MMAs of every fifth tile (a tile's MMAs form one dependent chain into its
// accumulator, so more issuers mean more chains in flight).  Two TMEM accumulators let
// the epilogue of one region overlap the MMAs of the next.  Every wait is bounded: on
// timeout the block sets the error flag, the other roles run out of their own waits, TMEM
// is freed and the block returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace vamrt {
namespace {

using namespace tc;

constexpr int kEpiSets = 2;         // epilogue warp sets of 4 (one per TMEM lane quarter)
constexpr int kLoadWarp0 = 4 * kEpiSets, kLoadWarps = 4, kMmaWarp0 = kLoadWarp0 + kLoadWarps, kMmaWarps = 5;
constexpr int kHaloThreads = 32 * (kMmaWarp0 + kMmaWarps);   // 8 epilogue, 4 loader, 5 MMA warps
constexpr int kPadX = 8;           // zero slots ahead of x = 0 in every staged row (x = -8 .. -1)
constexpr int kRowBytes = 32;      // one staged slot: 16 bf16 channels of one voxel
constexpr int kMaxTiles = 32;
constexpr int kSmemLimit = 225 * 1024;

struct HaloArgs {
    const __nv_bfloat16 *X, *Wt;
    const float *bias;
    void *Y;
    int *err;
    int D, H, W, Cin, Cout, relu;
    int TZ, TY, WP, PT, T, Nt;      // region planes / rows, slot pitches, M tiles, channels per item
    int NX, rowtile, mg, adv;       // dx taps per MMA; tile = one 128-voxel row; tile margin, advance
    int a_bytes, box_bytes, stage_bytes, ncols;   // staged input tile (with slack), its TMA bytes, stage
    int ry, nslice, nitems;         // regions along y, channel slices, work items
};

__device__ __forceinline__ int core_off(int r, int h) { return (r >> 3) * 256 + h * 128 + (r & 7) * 16; }

__device__ void halo_fail(volatile int *abort_flag, int *err)
{
    *abort_flag = 1;
    atomicExch(err, 1);
}

// raise the phase's expected transaction bytes (no arrival)
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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

// warps 4-7: per 16-channel chunk, one TMA box of the input tile (thread 0 adds its byte
// count to the stage's mbarrier before any arrival; the box's zero fill supplies every pad
// and out-of-volume halo voxel) and cp.async copies of the weights, into two stages
template <int TAPS>
__device__ void role_load(const CUtensorMap *xmap, const HaloArgs &a, uint32_t sbase, uint32_t full0,
                          uint32_t empty0, volatile int *abort_flag)
{
    constexpr int kHalo = TAPS == 27 ? 1 : 0;
    const int lt = threadIdx.x - kLoadWarp0 * 32, lane = lt & 31;
    const int nc = a.Cin >> 4;
    int i = 0;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int slice = item % a.nslice, r = item / a.nslice;
        const int z0 = (r / a.ry) * a.TZ - kHalo, y0 = (r % a.ry) * a.TY - kHalo, co0 = slice * a.Nt;
        for (int c = 0; c < nc; ++c, ++i) {
            const int s = i & 1;
            const uint32_t full = full0 + 8 * s, empty = empty0 + 8 * s;
            if (i >= 2) {
                const bool ok = mbar_wait(empty, ((i >> 1) - 1) & 1);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) halo_fail(abort_flag, a.err);
                    return;
                }
            }
            if (__any_sync(0xffffffffu, *abort_flag)) return;
            const uint32_t xs = sbase + s * a.stage_bytes;
            const uint32_t wb = xs + a.a_bytes;
            const int ng = TAPS * a.Nt * 2;
            for (int g = lt; g < ng; g += kLoadWarps * 32) {
                const int t = g / (2 * a.Nt), rem = g - t * 2 * a.Nt, co = rem >> 1, h = rem & 1;
                const int grp = t / a.NX, dxi = t - grp * a.NX;      // B rows n = dxi Nt + co
                cp_async16(wb + grp * a.NX * a.Nt * 32 + core_off(dxi * a.Nt + co, h),
                           a.Wt + (((int64_t)(co0 + co) * TAPS + t) * a.Cin + c * 16 + h * 8));
            }
            if (lt == 0) {
                mbar_expect_tx(full, (uint32_t)a.box_bytes);     // before this thread's own arrival
                tma_load_4d(xs, xmap, c * 16, -kPadX, y0, z0, full);
            }
            cp_async_wait_all();
            fence_proxy_async();
            mbar_arrive(full);
        }
    }
}

// lane 0 of MMA warp k: per staged chunk, one MMA per (tap group, tile) for tiles k, k + 4,
// ...  A tap group is the three dx taps of one (dz, dy): A is the slot run shifted by
// dz PT + dy WP, B stacks the three taps' weights in N (N = 3 Nt), and the epilogue adds
// the dx shift.  One thread keeps one MMA in flight at a time (about 90 ns each whatever N
// is), so four issuers and wide N are what bring the narrow layers of this network
// towards the tensor pipe's rate.
template <int TAPS>
__device__ void role_mma(const HaloArgs &a, int k0, uint32_t sbase, uint32_t tmem, const uint64_t *s_adesc,
                         uint32_t full0, uint32_t empty0, uint32_t accf0, uint32_t acce0, volatile int *abort_flag)
{
    const int nc = a.Cin >> 4, NN = a.NX * a.Nt, ngroups = TAPS / a.NX;
    const uint32_t idesc = instr_desc(128, NN);
    int i = 0, k = 0;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x, ++k) {
        const int b = k & 1;
        if (k >= 2 && !mbar_wait(acce0 + 8 * b, ((k >> 1) - 1) & 1)) {
            halo_fail(abort_flag, a.err);
            return;
        }
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(b * a.T * NN);
        for (int c = 0; c < nc; ++c, ++i) {
            const int s = i & 1;
            if (!mbar_wait(full0 + 8 * s, (i >> 1) & 1) || *abort_flag) {
                halo_fail(abort_flag, a.err);
                return;
            }
            tc_fence_after();
            const uint32_t wb = sbase + s * a.stage_bytes + a.a_bytes;
            for (int g = 0; g < ngroups; ++g) {
                int off = 0;
                if (TAPS == 27) off = (g / 3 - 1) * a.PT + (g % 3 - 1) * a.WP;
                // stage and (dz, dy) shift added to the descriptors' 16-byte address field
                const int64_t dt = (int64_t)(s * a.stage_bytes / 16 + off * (kRowBytes / 16));
                const uint64_t bdesc = smem_desc(wb + g * NN * 32, 128, 256);
                const uint32_t acc = (c | g) ? 1u : 0u;
                uint32_t d = dcol + (uint32_t)(k0 * NN);
                for (int j = k0; j < a.T; j += kMmaWarps, d += (uint32_t)(kMmaWarps * NN))
                    mma_bf16(d, (uint64_t)((int64_t)s_adesc[j] + dt), bdesc, idesc, acc);
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(accf0 + 8 * b);
    }
}

template <typename OT>
__device__ __forceinline__ void store16(OT *dst, const uint32_t *v, const float *bias, int relu)
{
    float r[16];
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
        const float4 b4 = bias ? __ldg((const float4 *)(bias + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
        r[i] = __uint_as_float(v[i]) + b4.x;
        r[i + 1] = __uint_as_float(v[i + 1]) + b4.y;
        r[i + 2] = __uint_as_float(v[i + 2]) + b4.z;
        r[i + 3] = __uint_as_float(v[i + 3]) + b4.w;
    }
    if (relu) {
#pragma unroll
        for (int i = 0; i < 16; ++i) r[i] = fmaxf(r[i], 0.f);
    }
    if constexpr (sizeof(OT) == 2) {
        uint32_t p[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
            p[i] = *(const uint32_t *)&h;
        }
        uint4 *d = (uint4 *)dst;
        d[0] = make_uint4(p[0], p[1], p[2], p[3]);
        d[1] = make_uint4(p[4], p[5], p[6], p[7]);
    } else {
        float4 *d = (float4 *)dst;
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
    }
}

// the 128 threads of epilogue set `set` (warps 4 set .. 4 set + 3) agree on a flag
// (named barrier 1 + set)
__device__ __forceinline__ bool epi_all(bool v, int set)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.b32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + set)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void epi_sync(int set) { asm volatile("bar.sync %0, 128;" ::"r"(1 + set) : "memory"); }

// warps 0-7: TMEM -> Y, two sets of four warps taking alternate tiles (warp 4 s + w of set
// s reads TMEM lane quarter w).  Row m of a tile holds, for each dx, the (dz, dy)-summed
// partial product of slot m; output slot m takes D[m - 1][dx = -1] + D[m][0] + D[m + 1][+1]
// (warp shuffles, and shared memory across the warps' 32-row boundaries).  Rows beyond a
// tile are pads (zero) for one-row tiles and are never outputs for margin tiles.
template <typename OT>
__device__ void role_epilogue(const HaloArgs &a, uint32_t tmem, const int *s_q, const int *s_oz, float *s_xch,
                              uint32_t accf0, uint32_t acce0, volatile int *abort_flag)
{
    const int set = threadIdx.x >> 7, tid = threadIdx.x & 127, warp = tid >> 5, lane = tid & 31;
    const int NN = a.NX * a.Nt;
    float *xch = s_xch + set * 256;
    int k = 0, step = 0;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x, ++k) {
        const int b = k & 1;
        const bool ok = mbar_wait(accf0 + 8 * b, (k >> 1) & 1) && !*abort_flag;
        if (!epi_all(ok, set)) {
            if (tid == 0) halo_fail(abort_flag, a.err);
            return;
        }
        tc_fence_after();
        const int slice = item % a.nslice, r = item / a.nslice;
        const int z0 = (r / a.ry) * a.TZ, y0 = (r % a.ry) * a.TY, co0 = slice * a.Nt;
        const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * a.T * NN);
        for (int j = set; j < a.T; j += kEpiSets) {
            const int q = s_q[j] + tid;
            const int oz = q >= 0 ? q / a.PT : -1, rem = q - oz * a.PT, oy = rem / a.WP, x = rem - oy * a.WP - kPadX;
            const int z = z0 + oz, y = y0 + oy;
            const bool valid = tid >= a.mg && tid < a.mg + a.adv && oz == s_oz[j] && oy < a.TY && x >= 0 &&
                               x < a.W && z < a.D && y < a.H;
            OT *dst = (OT *)a.Y + ((((int64_t)z * a.H + y) * a.W + x) * a.Cout + co0);
            for (int n0 = 0; n0 < a.Nt; n0 += 16, ++step) {
                const uint32_t col = lanes + (uint32_t)(j * NN + n0);
                uint32_t v[16];
                if (a.NX == 3) {
                    uint32_t dm[16], dp[16];
                    tmem_ld16_issue(col, dm);
                    tmem_ld16_issue(col + (uint32_t)a.Nt, v);
                    tmem_ld16_issue(col + (uint32_t)(2 * a.Nt), dp);
                    tmem_ld_wait();
                    // rows 32w - 1 and 32w + 32 live in the neighbouring warps: lane 31 of each
                    // warp publishes its dx = -1 part, lane 0 its dx = +1 part; every lane then
                    // reads both edges (broadcast) and selects without branching, so the
                    // shuffle loop has no divergent shared-memory loads to wait on
                    uint4 *xm = (uint4 *)(xch + (step & 1) * 128), *xp = xm + 16;   // [warp][4] x 16 B
                    if (lane == 31)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            xm[warp * 4 + i] = make_uint4(dm[4 * i], dm[4 * i + 1], dm[4 * i + 2], dm[4 * i + 3]);
                    if (lane == 0)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            xp[warp * 4 + i] = make_uint4(dp[4 * i], dp[4 * i + 1], dp[4 * i + 2], dp[4 * i + 3]);
                    epi_sync(set);
                    uint32_t el[16], er[16];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint4 l4 = warp > 0 ? xm[(warp - 1) * 4 + i] : make_uint4(0, 0, 0, 0);
                        const uint4 r4 = warp < 3 ? xp[(warp + 1) * 4 + i] : make_uint4(0, 0, 0, 0);
                        el[4 * i] = l4.x; el[4 * i + 1] = l4.y; el[4 * i + 2] = l4.z; el[4 * i + 3] = l4.w;
                        er[4 * i] = r4.x; er[4 * i + 1] = r4.y; er[4 * i + 2] = r4.z; er[4 * i + 3] = r4.w;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const uint32_t up = __shfl_up_sync(0xffffffffu, dm[i], 1);
                        const uint32_t dn = __shfl_down_sync(0xffffffffu, dp[i], 1);
                        const float left = __uint_as_float(lane == 0 ? el[i] : up);
                        const float right = __uint_as_float(lane == 31 ? er[i] : dn);
                        v[i] = __float_as_uint(left + __uint_as_float(v[i]) + right);
                    }
                } else {
                    tmem_ld16_issue(col, v);
                    tmem_ld_wait();
                }
                if (valid) store16<OT>(dst + n0, v, a.bias ? a.bias + co0 + n0 : nullptr, a.relu);
            }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * b);
    }
}

template <int TAPS, typename OT>
__global__ void __launch_bounds__(kHaloThreads, 1)
    conv3d_halo_kernel(const __grid_constant__ CUtensorMap xmap, const HaloArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[8];   // full[2], empty[2], acc_full[2], acc_empty[2]
    __shared__ uint32_t s_tmem;
    __shared__ int s_q[kMaxTiles], s_oz[kMaxTiles];
    __shared__ uint64_t s_adesc[kMaxTiles];
    __shared__ __align__(16) float s_xch[256 * kEpiSets];   // epilogue warp-boundary exchange, two buffers per set
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = smem_u32(smem);

    // first slot of each M tile (slot of the region's output voxel (0, 0, x) is x + kPadX),
    // and the output plane the tile belongs to (rows that run on into the next plane are
    // dropped); every start is a multiple of 8 slots, one 256-byte swizzle atom
    for (int j = tid; j < a.T; j += kHaloThreads) {
        int q, oz;
        if (a.rowtile) {          // W = 128: tile j is row (oz, oy), x = 0 .. 127
            oz = j / a.TY;
            q = oz * a.PT + (j - oz * a.TY) * a.WP + kPadX;
        } else {                  // runs through each plane's rows, advancing adv slots
            const int per_plane = (a.TY * a.WP + a.adv - 1) / a.adv;
            oz = j / per_plane;
            q = oz * a.PT + a.adv * (j - oz * per_plane);
        }
        s_q[j] = q;
        s_oz[j] = oz;
        // A operand of tile j at stage 0, centre tap: slot halo (PT + WP) + q, K-major with
        // 32-byte swizzled rows (layout type 6), 8-row groups 256 B apart
        s_adesc[j] = smem_desc(sbase + (uint32_t)((TAPS == 27 ? a.PT + a.WP : 0) + q) * kRowBytes, 16, 256) |
                     ((uint64_t)6 << 61);
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars[s]), kLoadWarps * 32);   // full: every loader thread (one with the box's bytes)
            mbar_init(smem_u32(&bars[2 + s]), kMmaWarps);     // empty: one commit per issuer
            mbar_init(smem_u32(&bars[4 + s]), kMmaWarps);     // accumulator full: likewise
            mbar_init(smem_u32(&bars[6 + s]), 4 * kEpiSets);   // accumulator empty: every epilogue warp
        }
        mbar_init_fence();
        s_abort = 0;
    }
    if (warp == kMmaWarp0) tmem_alloc(smem_u32(&s_tmem), (uint32_t)a.ncols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[2]);
    const uint32_t accf0 = smem_u32(&bars[4]), acce0 = smem_u32(&bars[6]);

    if (warp < kLoadWarp0)
        role_epilogue<OT>(a, tmem, s_q, s_oz, s_xch, accf0, acce0, &s_abort);
    else if (warp < kMmaWarp0)
        role_load<TAPS>(&xmap, a, sbase, full0, empty0, &s_abort);
    else if ((tid & 31) == 0)
        role_mma<TAPS>(a, warp - kMmaWarp0, sbase, tmem, s_adesc, full0, empty0, accf0, acce0, &s_abort);

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)a.ncols);
    }
}

// ---- host side ----

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace

// Region planner: choose (TZ, TY, Nt) minimising a simple model of the block time
// (max of tensor time and staging time per item, times the number of waves), subject to
// two stages fitting in shared memory and the accumulators in 512 TMEM columns.
// Returns false when the halo kernel cannot take the shape.
bool plan_conv3d_halo(int D, int H, int W, int Cin, int Cout, int taps, int sms, ConvHaloPlan *pl)
{
    if (W % 8 != 0 || Cin % 16 || Cout % 16 || Cout > 256 || sms < 1) return false;
    if (taps != 1 && taps != 27) return false;
    // rows of WP slots, x = -8 .. W + 7 (one TMA box dimension: at most 256); margin tiles
    // advance by whole 8-slot swizzle atoms
    const int halo = taps == 27 ? 1 : 0, NX = taps == 27 ? 3 : 1, WP = W + 2 * kPadX, nc = Cin / 16;
    if (WP > 256) return false;
    const int rowtile = W == 128, mg = (taps == 27 && !rowtile) ? 1 : 0, adv = mg ? 120 : 128;
    double best = 0.0;
    bool found = false;
    for (int Nt = Cout; Nt >= 16; Nt -= 16) {
        if (Cout % Nt || NX * Nt > 256) continue;
        for (int TZ = 1; TZ <= (D < 16 ? D : 16); ++TZ)
            for (int TY = 1; TY <= (H < 64 ? H : 64); ++TY) {
                const int PT = (TY + 2 * halo) * WP;
                const int64_t NSX = (int64_t)(TZ + 2 * halo) * PT;
                int T, qmax;
                if (rowtile) {
                    T = TZ * TY;
                    qmax = (TZ - 1) * PT + (TY - 1) * WP + kPadX;
                } else {
                    const int per = (TY * WP + adv - 1) / adv;
                    T = TZ * per;
                    qmax = (TZ - 1) * PT + (per - 1) * adv;
                }
                if (T > kMaxTiles || 2 * T * NX * Nt > 512) continue;     // two accumulators
                // rows past the TMA box (read only by discarded outputs) are slack
                const int64_t maxslot = halo * (PT + WP) + qmax + 127 + (halo ? PT + WP : 0);
                int64_t hs = NSX > maxslot + 1 ? NSX : maxslot + 1;
                hs = (hs + 7) / 8 * 8;
                const int64_t a_bytes = hs * kRowBytes;
                if (a_bytes >= (1 << 18)) continue;             // descriptor address range
                int64_t stage = a_bytes + (int64_t)taps * Nt * 32;
                stage = (stage + 1023) / 1024 * 1024;
                if (2 * stage > kSmemLimit) continue;
                // cycles per work item: an MMA into the accumulator of the issuer's previous
                // one waits about 470 cycles (in-kernel timers), independent ones (the issuer's
                // other tiles) issue about 175 cycles apart, and the pipe sustains about 11.5
                // cycles per 128 x 16 x 16; TMA boxes of 32-byte rows move about 40 B/cycle/SM;
                // an epilogue set takes about 2000 cycles per 16 channels of a tile, two sets
                // in parallel
                const double per_issuer = (double)((T + kMmaWarps - 1) / kMmaWarps) * 175.0;
                const double issue = per_issuer > 470.0 ? per_issuer : 470.0;
                const double pipe = (double)T * NX * Nt / 16.0 * 11.5;
                const double mma = (double)nc * (taps / NX) * (issue > pipe ? issue : pipe);
                const double load = (double)nc * stage / 40.0;
                const double epi = (double)T * Nt / 16.0 * 2000.0 / kEpiSets;
                double cost = mma > load ? mma : load;
                cost = (cost > epi ? cost : epi) + 500.0;
                const int64_t nreg = (int64_t)((D + TZ - 1) / TZ) * ((H + TY - 1) / TY) * (Cout / Nt);
                const double total = (double)((nreg + sms - 1) / sms) * cost;
                // ties go to the plan with more tiles: more issuers with a chain in flight
                if (!found || total < best || (total == best && T > pl->T)) {
                    found = true;
                    best = total;
                    int ncols = 32;
                    while (ncols < 2 * T * NX * Nt) ncols <<= 1;
                    pl->TZ = TZ; pl->TY = TY; pl->Nt = Nt; pl->T = T; pl->WP = WP; pl->PT = PT;
                    pl->NX = NX; pl->rowtile = rowtile; pl->mg = mg; pl->adv = adv;
                    pl->a_bytes = (int)a_bytes;
                    pl->box_bytes = (int)(NSX * kRowBytes);
                    pl->stage_bytes = (int)stage;
                    pl->ncols = ncols;
                    pl->ry = (H + TY - 1) / TY;
                    pl->nslice = Cout / Nt;
                    pl->nitems = (int)nreg;
                }
            }
    }
    return found;
}

cudaError_t launch_conv3d_halo(const void *X, const void *Wt, const float *bias, void *Y, int out_f32, int D, int H,
                               int W, int Cin, int Cout, int taps, int relu, int *err, cudaStream_t s)
{
    const int sms = sm_count();
    ConvHaloPlan pl;
    if (((uintptr_t)X & 15) || !plan_conv3d_halo(D, H, W, Cin, Cout, taps, sms, &pl)) return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc) return cudaErrorNotSupported;
    // the input tile of a region: box {16 channels, WP x from -8, TY (+ 2) rows, TZ (+ 2)
    // planes}, 32-byte swizzle, zero fill outside the volume
    const int halo = taps == 27 ? 1 : 0;
    CUtensorMap xmap;
    const cuuint64_t dims[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
    const cuuint64_t strides[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t box[4] = {16, (cuuint32_t)pl.WP, (cuuint32_t)(pl.TY + 2 * halo), (cuuint32_t)(pl.TZ + 2 * halo)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(X), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    HaloArgs a;
    a.X = (const __nv_bfloat16 *)X;
    a.Wt = (const __nv_bfloat16 *)Wt;
    a.bias = bias;
    a.Y = Y;
    a.err = err;
    a.D = D; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout; a.relu = relu;
    a.TZ = pl.TZ; a.TY = pl.TY; a.WP = pl.WP; a.PT = pl.PT; a.T = pl.T; a.Nt = pl.Nt;
    a.NX = pl.NX; a.rowtile = pl.rowtile; a.mg = pl.mg; a.adv = pl.adv;
    a.a_bytes = pl.a_bytes; a.box_bytes = pl.box_bytes; a.stage_bytes = pl.stage_bytes;
    a.ncols = pl.ncols;
    a.ry = pl.ry; a.nslice = pl.nslice; a.nitems = pl.nitems;
    // at least 116 KB of shared memory keeps one block per SM, so TMEM is never oversubscribed
    size_t smem = 2 * (size_t)pl.stage_bytes;
    if (smem < 116 * 1024) smem = 116 * 1024;
    const unsigned grid = (unsigned)(pl.nitems < sms ? pl.nitems : sms);
    cudaError_t e;
#define VAMRT_HALO(T, OT)                                                                                      \
    do {                                                                                                       \
        e = cudaFuncSetAttribute(conv3d_halo_kernel<T, OT>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 (int)smem);                                                                   \
        if (e == cudaSuccess) conv3d_halo_kernel<T, OT><<<grid, kHaloThreads, smem, s>>>(xmap, a);        \
    } while (0)
    if (taps == 27) {
        if (out_f32) VAMRT_HALO(27, float); else VAMRT_HALO(27, __nv_bfloat16);
    } else {
        if (out_f32) VAMRT_HALO(1, float); else VAMRT_HALO(1, __nv_bfloat16);
    }
#undef VAMRT_HALO
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vamrt
