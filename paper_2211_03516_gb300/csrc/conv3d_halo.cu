// Halo-tiled 3x3x3 (or 1x1x1) convolution on the 5th-generation tensor cores: a
// persistent, warp-specialised implicit GEMM whose input tiles arrive by TMA.
//
//   Y[p][co] = act( bias[co] + sum_{t, ci} X[p + off(t)][ci] * Wt[co][t][ci] )
//
// Same operation and layouts as conv3d_tc.cu (X [D][H][W][Cin] bf16, Wt [Cout][taps][Cin],
// Y [D][H][W][Cout] bf16 or fp32, zero padding); this kernel needs W % 8 == 0.
//
// Slot layout.  A work item is a region of TZ output planes x TY output rows x all W
// columns (and a slice of Nt output channels).  Its input tile -- (TZ + 2) planes x
// (TY + 2) rows with the one-voxel halo -- is staged one 16-channel chunk at a time as two
// 8-channel halves; each half is a run of 16-byte "slots" (8 bf16 channels of one voxel).
// A row takes WP = W + 8 slots: W voxels, then 8 zero slots, which are at once the x = W
// neighbour of this row and the x = -1 neighbour of the next (8 zero guard slots precede
// the first row).  The TMA writes this padding itself: X is described to it as a 5-D
// tensor (8 channels, 8 x, W / 8 x-groups, H, D) and the box asks for W / 8 + 1 x-groups,
// the last of which lies outside the tensor and is zero-filled, as are halo rows and
// planes outside the volume.
//
// GEMM mapping.  M = 128 consecutive slots of the region (TMEM lanes), N = Nt output
// channels (TMEM columns), K = 16 channels of one tap per MMA.  Because the slot index is
// linear in (z, y, x), the A operand of tap (dz, dy, dx) for a tile is the same slot run
// shifted by dz PT + dy WP + dx slots: one shared-memory descriptor per (tile, tap), no
// data movement.  A core matrix is 8 consecutive slots (128 contiguous bytes); SBO = 128 B,
// LBO = the distance between the two halves.  Tiles that start in padding or run past the
// region compute rows that the epilogue discards.  B (weights of one chunk, all taps) is
// staged by cp.async in the canonical K-major layout.
//
// Roles (192 threads): warps 0-3 drain TMEM (warp w owns lanes 32w..32w+31) and write Y;
// warp 4 issues the TMA and weight copies into two shared-memory stages; one thread of
// warp 5 issues the MMAs.  Two TMEM accumulators let the epilogue of one
// region overlap the MMAs of the next.  Every wait is bounded: on timeout the block sets
// the error flag, the other roles run out of their own waits, TMEM is freed and the
// block returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace vamrt {
namespace {

using namespace tc;

constexpr int kHaloThreads = 192;
constexpr int kGuard = 8;          // zero slots ahead of each staged half
constexpr int kMaxTiles = 32;
constexpr int kSmemLimit = 225 * 1024;

struct HaloArgs {
    const __nv_bfloat16 *Wt;
    const float *bias;
    void *Y;
    int *err;
    int D, H, W, Cin, Cout, relu;
    int TZ, TY, WP, PT, T, Nt;      // region planes / rows, slot pitches, M tiles, columns per item
    int half_bytes, x_bytes, stage_bytes, ncols;
    int ry, nslice, nitems;         // regions along y, channel slices, work items
};

__device__ __forceinline__ int core_off(int r, int h) { return (r >> 3) * 256 + h * 128 + (r & 7) * 16; }

__device__ void halo_fail(volatile int *abort_flag, int *err)
{
    *abort_flag = 1;
    atomicExch(err, 1);
}

// warp 4: TMA loads of the input halves and cp.async copies of the weights, two stages
template <int TAPS>
__device__ void role_load(const CUtensorMap *xmap, const HaloArgs &a, uint32_t sbase, uint32_t full0,
                          uint32_t empty0, volatile int *abort_flag)
{
    constexpr int kHalo = TAPS == 27 ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const int nc = a.Cin >> 4;
    int i = 0;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x) {
        const int slice = item % a.nslice, r = item / a.nslice;
        const int z0 = (r / a.ry) * a.TZ, y0 = (r % a.ry) * a.TY, co0 = slice * a.Nt;
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
            if (lane == 0) {
                mbar_expect_tx(full, 2u * a.x_bytes);
                tma_load_5d(xs + kGuard * 16, xmap, c * 16, 0, 0, y0 - kHalo, z0 - kHalo, full);
                tma_load_5d(xs + a.half_bytes + kGuard * 16, xmap, c * 16 + 8, 0, 0, y0 - kHalo, z0 - kHalo, full);
            }
            const uint32_t wb = xs + 2 * a.half_bytes;
            const int ng = TAPS * a.Nt * 2;
            for (int g = lane; g < ng; g += 32) {
                const int t = g / (2 * a.Nt), rem = g - t * 2 * a.Nt, co = rem >> 1, h = rem & 1;
                cp_async16(wb + t * a.Nt * 32 + core_off(co, h),
                           a.Wt + (((int64_t)(co0 + co) * TAPS + t) * a.Cin + c * 16 + h * 8));
            }
            cp_async_wait_all();
            fence_proxy_async();
            mbar_arrive(full);
        }
    }
}

// one thread of warp 5: T x TAPS MMAs per staged chunk
template <int TAPS>
__device__ void role_mma(const HaloArgs &a, uint32_t sbase, uint32_t tmem, const uint64_t *s_adesc, uint32_t full0,
                         uint32_t empty0, uint32_t accf0, uint32_t acce0, volatile int *abort_flag)
{
    const int nc = a.Cin >> 4;
    const uint32_t idesc = instr_desc(128, a.Nt);
    int i = 0, k = 0;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x, ++k) {
        const int b = k & 1;
        if (k >= 2 && !mbar_wait(acce0 + 8 * b, ((k >> 1) - 1) & 1)) {
            halo_fail(abort_flag, a.err);
            return;
        }
        tc_fence_after();
        const uint32_t dcol = tmem + (uint32_t)(b * a.T * a.Nt);
        for (int c = 0; c < nc; ++c, ++i) {
            const int s = i & 1;
            if (!mbar_wait(full0 + 8 * s, (i >> 1) & 1) || *abort_flag) {
                halo_fail(abort_flag, a.err);
                return;
            }
            tc_fence_after();
            const uint32_t wb = sbase + s * a.stage_bytes + 2 * a.half_bytes;
            for (int t = 0; t < TAPS; ++t) {
                int off = 0;
                if (TAPS == 27) off = (t / 9 - 1) * a.PT + ((t / 3) % 3 - 1) * a.WP + (t % 3 - 1);
                // stage and tap shift added to the descriptors' 16-byte address field
                const int64_t dt = (int64_t)(s * a.stage_bytes / 16 + off);
                const uint64_t bdesc = smem_desc(wb + t * a.Nt * 32, 128, 256);
                const uint32_t acc = (c | t) ? 1u : 0u;
                uint32_t d = dcol;
                for (int j = 0; j < a.T; ++j, d += (uint32_t)a.Nt)
                    mma_bf16(d, (uint64_t)((int64_t)s_adesc[j] + dt), bdesc, idesc, acc);
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(accf0 + 8 * b);
    }
}

template <typename OT>
__device__ __forceinline__ void store16(OT *dst, const float *v, const float *bias, int relu)
{
    float r[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        r[i] = v[i] + (bias ? bias[i] : 0.f);
        if (relu) r[i] = fmaxf(r[i], 0.f);
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

// warps 0-3: TMEM -> bias, activation -> Y
template <typename OT>
__device__ void role_epilogue(const HaloArgs &a, uint32_t tmem, const int *s_q, const int *s_oz, uint32_t accf0,
                              uint32_t acce0, volatile int *abort_flag)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int k = 0;
    for (int item = blockIdx.x; item < a.nitems; item += gridDim.x, ++k) {
        const int b = k & 1;
        const bool ok = mbar_wait(accf0 + 8 * b, (k >> 1) & 1);
        if (!__all_sync(0xffffffffu, ok) || __any_sync(0xffffffffu, *abort_flag)) {
            if (lane == 0) halo_fail(abort_flag, a.err);
            return;
        }
        tc_fence_after();
        const int slice = item % a.nslice, r = item / a.nslice;
        const int z0 = (r / a.ry) * a.TZ, y0 = (r % a.ry) * a.TY, co0 = slice * a.Nt;
        const uint32_t lanes = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * a.T * a.Nt);
        for (int j = 0; j < a.T; ++j) {
            const int q = s_q[j] + tid;
            const int oz = q / a.PT, rem = q - oz * a.PT, oy = rem / a.WP, x = rem - oy * a.WP;
            const int z = z0 + oz, y = y0 + oy;
            const bool valid = oz == s_oz[j] && oy < a.TY && x < a.W && z < a.D && y < a.H;
            OT *dst = (OT *)a.Y + ((((int64_t)z * a.H + y) * a.W + x) * a.Cout + co0);
            for (int n0 = 0; n0 < a.Nt; n0 += 16) {
                float v[16];
                tmem_ld16(lanes + (uint32_t)(j * a.Nt + n0), v);
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
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = smem_u32(smem);

    // guard slots: the x = -1 neighbours of each staged half's first row, zero for the launch
    for (int i = tid; i < 2 * 2 * kGuard; i += kHaloThreads) {
        const int s = i / (2 * kGuard), h = (i / kGuard) & 1, g = i % kGuard;
        *(uint4 *)(smem + s * a.stage_bytes + h * a.half_bytes + g * 16) = make_uint4(0, 0, 0, 0);
    }
    // first slot of each M tile, relative to output voxel (0, 0, 0) of the region, and the
    // output plane the tile belongs to (rows that run on into the next plane are dropped)
    for (int j = tid; j < a.T; j += kHaloThreads) {
        int q, oz;
        if (a.W % 128 == 0) {     // tiles never straddle a row
            const int per_row = a.W / 128, per_plane = a.TY * per_row;
            oz = j / per_plane;
            const int r = j - oz * per_plane, oy = r / per_row;
            q = oz * a.PT + oy * a.WP + 128 * (r - oy * per_row);
        } else {                  // consecutive runs of 128 slots through each plane's rows
            const int per_plane = (a.TY * a.WP + 127) / 128;
            oz = j / per_plane;
            q = oz * a.PT + 128 * (j - oz * per_plane);
        }
        s_q[j] = q;
        s_oz[j] = oz;
        // A operand of tile j at stage 0, centre tap: slot kGuard + halo (PT + WP) + q
        s_adesc[j] = smem_desc(sbase + (uint32_t)(kGuard + (TAPS == 27 ? a.PT + a.WP : 0) + q) * 16,
                               (uint32_t)a.half_bytes, 128);
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars[s]), 32);         // full: 32 loader lanes (+ TMA bytes)
            mbar_init(smem_u32(&bars[2 + s]), 1);      // empty: one MMA commit
            mbar_init(smem_u32(&bars[4 + s]), 1);      // accumulator full: one MMA commit
            mbar_init(smem_u32(&bars[6 + s]), 4);      // accumulator empty: 4 epilogue warps
        }
        mbar_init_fence();
        s_abort = 0;
    }
    if (warp == 5) tmem_alloc(smem_u32(&s_tmem), (uint32_t)a.ncols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[2]);
    const uint32_t accf0 = smem_u32(&bars[4]), acce0 = smem_u32(&bars[6]);

    if (warp < 4)
        role_epilogue<OT>(a, tmem, s_q, s_oz, accf0, acce0, &s_abort);
    else if (warp == 4)
        role_load<TAPS>(&xmap, a, sbase, full0, empty0, &s_abort);
    else if ((tid & 31) == 0)
        role_mma<TAPS>(a, sbase, tmem, s_adesc, full0, empty0, accf0, acce0, &s_abort);

    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)a.ncols);
    }
}

// ---- host side ----

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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
    if (W % 8 != 0 || W / 8 + 1 > 256 || Cin % 16 || Cout % 16 || Cout > 256 || sms < 1) return false;
    if (taps != 1 && taps != 27) return false;
    if (!encode_fn()) return false;           // driver without TMA descriptor encoding
    const int halo = taps == 27 ? 1 : 0, WP = W + 8, nc = Cin / 16;
    double best = 0.0;
    bool found = false;
    for (int Nt = Cout; Nt >= 16; Nt -= 16) {
        if (Cout % Nt) continue;
        for (int TZ = 1; TZ <= (D < 16 ? D : 16); ++TZ)
            for (int TY = 1; TY <= (H < 64 ? H : 64); ++TY) {
                if (TY + 2 * halo > 256 || TZ + 2 * halo > 256) continue;
                const int PT = (TY + 2 * halo) * WP;
                const int64_t NSX = (int64_t)(TZ + 2 * halo) * PT;
                int T, qmax;
                if (W % 128 == 0) {
                    T = TZ * TY * (W / 128);
                    qmax = (TZ - 1) * PT + (TY - 1) * WP + W - 128;
                } else {
                    const int per = (TY * WP + 127) / 128;
                    T = TZ * per;
                    qmax = (TZ - 1) * PT + (per - 1) * 128;
                }
                if (T > kMaxTiles || 2 * T * Nt > 512) continue;     // two accumulators
                const int64_t maxslot = kGuard + halo * (PT + WP) + qmax + 127 + (halo ? PT + WP + 1 : 0);
                int64_t hs = kGuard + NSX > maxslot + 1 ? kGuard + NSX : maxslot + 1;
                hs = (hs + 7) / 8 * 8;
                const int64_t half_bytes = hs * 16;
                if (half_bytes >= (1 << 18)) continue;          // descriptor LBO / address range
                int64_t stage = 2 * half_bytes + (int64_t)taps * Nt * 32;
                stage = (stage + 1023) / 1024 * 1024;
                if (2 * stage > kSmemLimit) continue;
                const double mma = (double)nc * taps * T * Nt / 16.0 * 8.5;
                const double load = (double)nc * stage / 64.0;
                const double cost = (mma > load ? mma : load) + 300.0;
                const int64_t nreg = (int64_t)((D + TZ - 1) / TZ) * ((H + TY - 1) / TY) * (Cout / Nt);
                const double total = (double)((nreg + sms - 1) / sms) * cost;
                if (!found || total < best) {
                    found = true;
                    best = total;
                    int ncols = 32;
                    while (ncols < 2 * T * Nt) ncols <<= 1;
                    pl->TZ = TZ; pl->TY = TY; pl->Nt = Nt; pl->T = T; pl->WP = WP; pl->PT = PT;
                    pl->half_bytes = (int)half_bytes;
                    pl->x_bytes = (int)(16 * (int64_t)WP * (TY + 2 * halo) * (TZ + 2 * halo));
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
    if (!plan_conv3d_halo(D, H, W, Cin, Cout, taps, sms, &pl)) return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    const int halo = taps == 27 ? 1 : 0;
    CUtensorMap map;
    const cuuint64_t dims[5] = {(cuuint64_t)Cin, 8, (cuuint64_t)(W / 8), (cuuint64_t)H, (cuuint64_t)D};
    const cuuint64_t strides[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)Cin * 16, (cuuint64_t)W * Cin * 2,
                                   (cuuint64_t)H * W * Cin * 2};
    const cuuint32_t box[5] = {8, 8, (cuuint32_t)(W / 8 + 1), (cuuint32_t)(pl.TY + 2 * halo),
                               (cuuint32_t)(pl.TZ + 2 * halo)};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(X), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    HaloArgs a;
    a.Wt = (const __nv_bfloat16 *)Wt;
    a.bias = bias;
    a.Y = Y;
    a.err = err;
    a.D = D; a.H = H; a.W = W; a.Cin = Cin; a.Cout = Cout; a.relu = relu;
    a.TZ = pl.TZ; a.TY = pl.TY; a.WP = pl.WP; a.PT = pl.PT; a.T = pl.T; a.Nt = pl.Nt;
    a.half_bytes = pl.half_bytes; a.x_bytes = pl.x_bytes; a.stage_bytes = pl.stage_bytes;
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
        if (e == cudaSuccess) conv3d_halo_kernel<T, OT><<<grid, kHaloThreads, smem, s>>>(map, a);              \
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
