// The two hot operators: projection (adjoint A^T, a gather) and dose (forward A, a
// scatter), sharing one tiled traversal.
//
// Work mapping.  A block owns 8 x 32 pixels (8 columns u, one warp per column running
// down 32 rows v) of one angle; a thread owns one pixel and walks its aperture rays one
// after the other.  For a given aperture sample the block's 256 rays form a coherent
// bundle, so the block
// advances them together in chunks: chunk c holds the samples whose position on the
// theta = 0 frame's y axis (the projection direction) lies in [y0 + 16 c, y0 + 16 (c+1))
// voxels.  For each chunk the block
//   1. takes the union of its rays' trilinear footprints (an axis-aligned box of voxels,
//      x rounded out to 16-byte groups),
//   2. adjoint: stages that box of the volume into shared memory with 16-byte loads;
//      forward: zeroes a shared-memory accumulator of that box,
//   3. walks the samples: 8 shared-memory reads (adjoint) or 8 shared-memory atomic adds
//      (forward) per sample,
//   4. forward: flushes the box with 16-byte vector reductions (red.global.add.v4.f32)
//      into the FP32 dose accumulator, skipping all-zero groups.
// The global memory system thus sees about one coalesced access per box voxel per chunk
// instead of 8 scattered accesses per sample, and the dose accumulator receives sums of
// about ten samples per voxel and chunk instead of single samples.  A chunk whose box
// does not fit in shared memory (unusually divergent bundles) is walked directly on
// global memory with the same arithmetic.
//
// Sample positions.  Per ray and angle the entry point and direction are rotated into the
// vial frame in FP64 and converted to Q32.32 fixed point, sample j at q0 + j * step.
// Inside a box a chunk is walked backwards from its last sample, whose Q32.32 position is
// cut to a 32-bit Q9.23 offset from the box origin, by the step cut to Q9.23 (one 32-bit
// add per axis and sample; the drift stays below 2^-23 voxel per sample and resets every
// chunk).  Walking backwards lets the Beer-Lambert factor enter by Horner's rule (one
// fused multiply-add per sample).  Positions are linear in j, so the cells a chunk visits
// lie between the cells of its two end positions, which the box is built from.
//
// Grid order.  Blocks are launched pixel-column tile fastest, then angle, then pixel-row
// tile, so the blocks resident together share a row tile: one slab of z planes of the
// volume (and one band of the ray table), which stays in L2 while every angle passes
// over it -- volumes far larger than L2 are then read from HBM about once per row tile.
//
// The caller's volume is copied into a scratch volume with one voxel of zero halo (zero
// padding outside the grid, Sec. 2.2's weights then need no bounds tests).  Each ray's
// sample range is trimmed once so that every sample's cell lies inside the padded grid.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>

#include <type_traits>

#include "internal.cuh"

namespace vamrt {
namespace {

constexpr double kFix = 4294967296.0;  // 2^32
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ void st_val(float *p, float x) { *p = x; }
__device__ __forceinline__ void st_val(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ void st_val(__half *p, float x) { *p = __float2half_rn(x); }

__device__ __forceinline__ float bf16_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// four consecutive voxels starting at a 4-aligned element (16 B for FP32, 8 B for BF16)
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p)
{
    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
    return make_float4(bf16_lo(w.x), bf16_hi(w.x), bf16_lo(w.y), bf16_hi(w.y));
}
__device__ __forceinline__ float4 ld4(const __half *p)
{
    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&w.x));
    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&w.y));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}
__device__ __forceinline__ float ld1(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __nv_bfloat16 *p)
{
    return __uint_as_float(((unsigned)__ldg(reinterpret_cast<const unsigned short *>(p))) << 16);
}
__device__ __forceinline__ float ld1(const __half *p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ void red_v4(float *p, float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// ---------------------------------------------------------------------------------
// halo copy: scratch[zp][yp][xp] = vol[zp-1][yp-1][xp-1] inside, 0 elsewhere
// ---------------------------------------------------------------------------------
template <typename VT>
__global__ void pad_kernel(const VT *__restrict__ vol, VT *__restrict__ out, int nx, int ny, int nz, int px,
                           int py, int64_t total)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int xp = (int)(i % px);
        const int yp = (int)((i / px) % py);
        const int zp = (int)(i / ((int64_t)px * py));
        VT val = VT(0.0f);
        if (xp >= 1 && xp <= nx && yp >= 1 && yp <= ny && zp >= 1 && zp <= nz)
            val = vol[((int64_t)(zp - 1) * ny + (yp - 1)) * nx + (xp - 1)];
        out[i] = val;
    }
}

// dose[z][y][x] (+)= scratch[z+1][y+1][x+1]
template <typename DT>
__global__ void unpad_kernel(const float *__restrict__ acc, DT *__restrict__ dose, int nx, int ny, int nz, int px,
                             int py, int accumulate)
{
    const int64_t total = (int64_t)nx * ny * nz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        float val = acc[((int64_t)(z + 1) * py + (y + 1)) * px + (x + 1)];
        if (accumulate) val += to_f(dose[i]);
        st_val(dose + i, val);
    }
}

// ---------------------------------------------------------------------------------
// per-ray state
// ---------------------------------------------------------------------------------
struct Ray {
    long long q0x, q0y, q0z;  // Q32.32 position of sample 0
    long long sx, sy, sz;     // Q32.32 advance per sample
    float att;                // log2 of the Beer-Lambert factor per sample
    float w;                  // T1 T2 delta_mm / M
    float ey, dy;             // theta = 0 frame: y(j) = ey + (j + 1/2) dy (voxels)
    float inv_dy;             // 1 / dy
    int d23x, d23y, d23z;     // the advance rounded to Q9.23 (box walks)
    int jlo, jhi;
};

// the Q32.32 step rounded to Q9.23 (any fixed integer step keeps the walk linear in j)
__device__ __forceinline__ long long step23(long long s) { return (s + 256) >> 9; }

// Q32.32 z of sample j lies in [0, pz - 1): its cell and the cell above are inside the
// padded grid.
__device__ __forceinline__ bool z_inside(const OpParams &P, const Ray &R, int j)
{
    const long long qz = R.q0z + (long long)j * R.sz;
    return qz >= 0 && qz < ((long long)(P.pz - 1) << 32);
}

__device__ __forceinline__ bool ray_begin(const OpParams &P, int64_t r, double2 cs, Ray &R, bool unattenuated)
{
    const int2 J = P.J[r];
    if (J.x >= J.y) return false;
    const double4_32a A = P.A[r], B = P.B[r];
    const double c = cs.x, s = cs.y;
    const double ex = A.x, ey = A.y, dl = A.w;
    const double stx = (c * B.x - s * B.y) * dl;
    const double sty = (s * B.x + c * B.y) * dl;
    const double stz = B.z * dl;
    // sample 0 sits half a step inside the entry point
    const double q0x = P.cx + (c * ex - s * ey) + 0.5 * stx;
    const double q0y = P.cy + (s * ex + c * ey) + 0.5 * sty;
    const double q0z = P.cz + A.z + 0.5 * stz;
    R.q0x = __double2ll_rn(q0x * kFix);
    R.q0y = __double2ll_rn(q0y * kFix);
    R.q0z = __double2ll_rn(q0z * kFix);
    R.sx = __double2ll_rn(stx * kFix);
    R.sy = __double2ll_rn(sty * kFix);
    R.sz = __double2ll_rn(stz * kFix);
    // the paper-literal projection (Sec. 2.4): no Beer-Lambert or Fresnel factor, weight delta / M
    R.att = unattenuated ? 0.f : P.neg_mu_vox_log2e * (float)A.w;
    R.w = unattenuated ? (float)A.w * P.h_over_m : (float)B.w;
    R.ey = (float)A.y;
    R.dy = (float)(A.w * B.y);
    R.inv_dy = 1.0f / R.dy;
    R.d23x = (int)step23(R.sx);
    R.d23y = (int)step23(R.sy);
    R.d23z = (int)step23(R.sz);
    // The traced sample range [j_lo, j_hi) keeps -1 < q_z < nz in FP64; the FP32 table's
    // rounding can put an end sample a hair outside.  Drop such end samples (their
    // in-grid weight is ~1e-5 of a sample's) so that no sample needs a clamp later.
    int jlo = J.x, jhi = J.y;
    for (int t = 0; t < 4 && jlo < jhi && !z_inside(P, R, jlo); ++t) ++jlo;
    for (int t = 0; t < 4 && jlo < jhi && !z_inside(P, R, jhi - 1); ++t) --jhi;
    if (jlo < jhi && !(z_inside(P, R, jlo) && z_inside(P, R, jhi - 1))) jhi = jlo;   // never for valid tables
    R.jlo = jlo;
    R.jhi = jhi;
    return jlo < jhi;
}

// rays that hardly advance along y are taken whole in their first chunk
constexpr float kMinDy = 1e-4f;

__device__ __forceinline__ int chunk_of(const OpParams &P, const Ray &R, int j)
{
    const float y = fmaf((float)j + 0.5f, R.dy, R.ey);
    return (int)floorf((y - P.y0) * (1.0f / kChunkVox));
}

// First sample whose y lies at or beyond the boundary at half-chunk h, i.e. at
// y0 + h * kChunkVox / 2 (monotone in h).  Chunk c spans half-chunks 2c and 2c + 1; a
// chunk whose box does not fit is walked as its two halves.
__device__ __forceinline__ int half_start(const OpParams &P, const Ray &R, int h)
{
    const float yc = P.y0 + (float)(h * (kChunkVox / 2));
    const float j = ceilf((yc - R.ey) * R.inv_dy - 0.5f);
    return (int)fminf(fmaxf(j, (float)R.jlo), (float)R.jhi);
}

// Samples [jl, jh) of half-chunks [h0, h1) of a ray whose samples span chunks cmin..cmax.
__device__ __forceinline__ void range_samples(const OpParams &P, const Ray &R, int h0, int h1, int cmin, int cmax,
                                              int &jl, int &jh)
{
    if (!(R.dy > kMinDy)) {
        jl = (h0 == 2 * cmin) ? R.jlo : R.jhi;
        jh = R.jhi;
        return;
    }
    jl = (h0 == 2 * cmin) ? R.jlo : half_start(P, R, h0);
    jh = (h1 == 2 * cmax + 2) ? R.jhi : half_start(P, R, h1);
}

struct Cell {
    int ix, iy, iz;
    float fx, fy, fz;
};

__device__ __forceinline__ float frac32(long long q)
{
    // top 23 fraction bits as a float in [0, 1), exactly
    return __uint_as_float(0x3f800000u | ((unsigned)q >> 9)) - 1.0f;
}

// Cell of a sample at an absolute Q32.32 position (inside the padded grid: z by the ray's
// sample range, x and y because the grid encloses the resin cylinder with a margin).
__device__ __forceinline__ Cell cell_of(long long qx, long long qy, long long qz)
{
    Cell c;
    c.ix = (int)(qx >> 32);
    c.iy = (int)(qy >> 32);
    c.iz = (int)(qz >> 32);
    c.fx = frac32(qx);
    c.fy = frac32(qy);
    c.fz = frac32(qz);
    return c;
}

// i / d for 0 <= i < 2^22 - 1 and d >= 1 through an FP32 reciprocal: (i + 1/2) / d lies at
// least 1/(2d) from an integer, while the reciprocal and the product together are off by
// less than (i + 1/2) / d * 2^-23 < 1/(2d).
__device__ __forceinline__ int fdiv(int i, float inv_d) { return (int)(((float)i + 0.5f) * inv_d); }

// A box is visited as slots (pixel row yy, 16-byte group x4) of a z plane, ey * ex4 of
// them, each slot walked down the planes by a pointer increment.  Thread t takes the items
// t, t + kThreads, ...: when a plane has fewer slots than the block has threads, the
// planes are dealt out in `phases` interleaved sets, one item per (set, slot).
struct SlotWalk {
    int slots, phases, items;
    float inv_slots, inv_ex4;
    __device__ __forceinline__ SlotWalk(int ex4, int ey)
    {
        slots = ex4 * ey;
        phases = max(1, kThreads / slots);
        items = phases * slots;
        inv_slots = 1.0f / (float)slots;
        inv_ex4 = 1.0f / (float)ex4;
    }
    // item -> first plane zp, row yy, group x4
    __device__ __forceinline__ void at(int it, int ex4, int &zp, int &yy, int &x4) const
    {
        zp = fdiv(it, inv_slots);
        const int s = it - zp * slots;
        yy = fdiv(s, inv_ex4);
        x4 = s - yy * ex4;
    }
};

// Packed FP32 pairs (sm_100 family): one instruction performs two independent
// round-to-nearest operations, so the results are bit-identical to the scalar forms while
// the issue-bound sample loops spend fewer instructions.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ void upk2i(f32x2 v, int &lo, int &hi) { asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(v)); }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Trilinear value at a cell from its 8 corners (x-lerps of the z = 0 and z = 1 corners
// in pairs, then the y-lerps, then z).
__device__ __forceinline__ float trilerp(float fx, float fy, float fz, float v000, float v100, float v010, float v110,
                                         float v001, float v101, float v011, float v111)
{
    const f32x2 fx2 = pk2(fx, fx);
    const f32x2 a0 = pk2(v000, v001), a1 = pk2(v010, v011);
    const f32x2 x0 = fma2(fx2, sub2(pk2(v100, v101), a0), a0);   // (x00, x01)
    const f32x2 x1 = fma2(fx2, sub2(pk2(v110, v111), a1), a1);   // (x10, x11)
    float y0, y1;
    upk2(fma2(pk2(fy, fy), sub2(x1, x0), x0), y0, y1);
    return fmaf(fz, y1 - y0, y0);
}

// ---- global-memory walks (chunks whose box does not fit in shared memory) ----------
// Beer-Lambert factor of samples jl, jl+1, ...: exact exp2 at the start of each run,
// then one multiply per sample.
template <typename VT>
__device__ __noinline__ float walk_gather_global(const OpParams &P, const Ray &R, int jl, int jh, const VT *vol)
{
    long long qx = R.q0x + (long long)jl * R.sx;
    long long qy = R.q0y + (long long)jl * R.sy;
    long long qz = R.q0z + (long long)jl * R.sz;
    const int sx = P.px, sxy = P.px * P.py;
    float att = exp2f(R.att * ((float)jl + 0.5f));
    const float ratio = exp2f(R.att);
    float acc = 0.f;
    for (int j = jl; j < jh; ++j) {
        const Cell c = cell_of(qx, qy, qz);
        const VT *p = vol + (c.iz * sxy + c.iy * sx + c.ix);
        const float val = trilerp(c.fx, c.fy, c.fz, ld1(p), ld1(p + 1), ld1(p + sx), ld1(p + sx + 1), ld1(p + sxy),
                                  ld1(p + sxy + 1), ld1(p + sxy + sx), ld1(p + sxy + sx + 1));
        acc = fmaf(att, val, acc);
        att *= ratio;
        qx += R.sx;
        qy += R.sy;
        qz += R.sz;
    }
    return acc;
}

// The 8 trilinear shares of weight w at a cell.
struct Shares {
    float s000, s100, s010, s110, s001, s101, s011, s111;
};
__device__ __forceinline__ Shares shares(float w, const Cell &c)
{
    const float wz1 = w * c.fz, wz0 = w - wz1;
    const float w01 = wz0 * c.fy, w00 = wz0 - w01;
    const float w11 = wz1 * c.fy, w10 = wz1 - w11;
    Shares S;
    S.s100 = w00 * c.fx; S.s000 = w00 - S.s100;
    S.s110 = w01 * c.fx; S.s010 = w01 - S.s110;
    S.s101 = w10 * c.fx; S.s001 = w10 - S.s101;
    S.s111 = w11 * c.fx; S.s011 = w11 - S.s111;
    return S;
}

// FP32 reductions straight into the padded accumulator.
__device__ __noinline__ void walk_scatter_global(const OpParams &P, const Ray &R, int jl, int jh, float wray,
                                                 float *dst)
{
    long long qx = R.q0x + (long long)jl * R.sx;
    long long qy = R.q0y + (long long)jl * R.sy;
    long long qz = R.q0z + (long long)jl * R.sz;
    const int sx = P.px, sxy = P.px * P.py;
    float att = exp2f(R.att * ((float)jl + 0.5f));
    const float ratio = exp2f(R.att);
    for (int j = jl; j < jh; ++j) {
        const Cell c = cell_of(qx, qy, qz);
        float *p = dst + (c.iz * sxy + c.iy * sx + c.ix);
        const Shares S = shares(wray * att, c);
        atomicAdd(p, S.s000);
        atomicAdd(p + 1, S.s100);
        atomicAdd(p + sx, S.s010);
        atomicAdd(p + sx + 1, S.s110);
        atomicAdd(p + sxy, S.s001);
        atomicAdd(p + sxy + 1, S.s101);
        atomicAdd(p + sxy + sx, S.s011);
        atomicAdd(p + sxy + sx + 1, S.s111);
        att *= ratio;
        qx += R.sx;
        qy += R.sy;
        qz += R.sz;
    }
}

// ---- shared-memory walks ------------------------------------------------------------
// Inside a box the walk runs backwards, from the chunk's last sample jh-1 (anchored
// exactly: its Q32.32 position cut to Q9.23 relative to the box origin) down to jl,
// stepping by the ray's advance rounded to Q9.23.  All positions are then a linear
// integer function of j, so the cells they visit lie between the cells of the two end
// positions, which the box is built from (chunk_bounds computes the far end exactly as
// the walk reaches it).  The truncated step drifts by < 2^-23 voxel per sample.
struct Q23 {
    int x, y, z;
};


// Absolute Q9.23 position of a chunk's last sample jh-1: the walk's exact anchor.
struct Anchor {
    long long x, y, z;
};
__device__ __forceinline__ Anchor anchor_at(const Ray &R, int jh)
{
    const long long j1 = jh - 1;
    return Anchor{(R.q0x + j1 * R.sx) >> 9, (R.q0y + j1 * R.sy) >> 9, (R.q0z + j1 * R.sz) >> 9};
}

__device__ __forceinline__ float frac23(int q) { return __uint_as_float(0x3f800000u | ((unsigned)q & 0x7fffffu)) - 1.0f; }

// Gather over samples jh-1 down to jl, Horner form: returns sum_j r^(j - jl) v_j,
// r = the Beer-Lambert factor per sample (the caller multiplies by r^(jl + 1/2)).
__device__ __forceinline__ float walk_gather_box(const Ray &R, const Anchor &an, int jl, int jh, int ox, int oy,
                                                 int oz, const float *box, int sx, int sxy)
{
    int qx = (int)(an.x - ((long long)ox << 23));
    int qy = (int)(an.y - ((long long)oy << 23));
    int qz = (int)(an.z - ((long long)oz << 23));
    const int dx = R.d23x, dy = R.d23y, dz = R.d23z;
    const float ratio = exp2f(R.att);
    float acc = 0.f;
#pragma unroll 2
    for (int j = jh - 1; j >= jl; --j) {
        const int b = (qz >> 23) * sxy + (qy >> 23) * sx + (qx >> 23);
        const float *p = box + b;
        const float val = trilerp(frac23(qx), frac23(qy), frac23(qz), p[0], p[1], p[sx], p[sx + 1], p[sxy],
                                  p[sxy + 1], p[sxy + sx], p[sxy + sx + 1]);
        acc = fmaf(acc, ratio, val);
        qx -= dx;
        qy -= dy;
        qz -= dz;
    }
    return acc;
}

// Shared-memory box: fixed-point integer accumulation.  Shared-memory integer atomics
// are native, FP32 ones are not.  `scale` maps the largest ray weight of the block to
// well under 2^22, and the bound on shares per voxel and chunk keeps every box sum below
// 2^31.  A share x becomes the integer round(x) in one of two ways:
//   - any sign: x + 1.5 * 2^23 holds round(x) + 0x4B400000 in its bit pattern (|x| < 2^22),
//     the offset subtracted before the atomic;
//   - x >= 0 (warps whose rays all carry non-negative weights, as the optimiser's clamped
//     projections do): x * 2^-149 is the subnormal whose bit pattern is round(x) itself
//     (x < 2^23), so no subtraction is needed.
// Both round to nearest, ties to even: the box sums are identical.
template <bool kNonNeg>
__device__ __forceinline__ void walk_scatter_box(const Ray &R, const Anchor &an, int jl, int jh, float wray,
                                                 float scale, int ox, int oy, int oz, int *box, int sx, int sxy)
{
    int qx = (int)(an.x - ((long long)ox << 23));
    int qy = (int)(an.y - ((long long)oy << 23));
    int qz = (int)(an.z - ((long long)oz << 23));
    const int dx = R.d23x, dy = R.d23y, dz = R.d23z;
    // weight of sample jh-1, then one division by the per-sample factor per step down
    float w = wray * scale * exp2f(R.att * ((float)(jh - 1) + 0.5f));
    const float inv_ratio = exp2f(-R.att);
    const f32x2 conv = kNonNeg ? pk2(0x1p-149f, 0x1p-149f) : pk2(12582912.0f, 12582912.0f);
    const int bias = kNonNeg ? 0 : 0x4B400000;
#pragma unroll 8
    for (int j = jh - 1; j >= jl; --j) {
        const float fx = frac23(qx), fy = frac23(qy), fz = frac23(qz);
        int *p = box + ((qz >> 23) * sxy + (qy >> 23) * sx + (qx >> 23));
        // the eight shares in pairs (z = 0, z = 1), then to fixed point
        const float wz1 = w * fz, wz0 = w - wz1;
        const f32x2 fx2 = pk2(fx, fx);
        const f32x2 z = pk2(wz0, wz1);
        const f32x2 w1 = mul2(z, pk2(fy, fy));             // (w01, w11)
        const f32x2 w0 = sub2(z, w1);                      // (w00, w10)
        const f32x2 s1a = mul2(w0, fx2), s1b = mul2(w1, fx2);   // (s100, s101), (s110, s111)
        int i000, i001, i100, i101, i010, i011, i110, i111;
        if (kNonNeg) {
            upk2i(mul2(sub2(w0, s1a), conv), i000, i001);
            upk2i(mul2(s1a, conv), i100, i101);
            upk2i(mul2(sub2(w1, s1b), conv), i010, i011);
            upk2i(mul2(s1b, conv), i110, i111);
        } else {
            upk2i(add2(sub2(w0, s1a), conv), i000, i001);
            upk2i(add2(s1a, conv), i100, i101);
            upk2i(add2(sub2(w1, s1b), conv), i010, i011);
            upk2i(add2(s1b, conv), i110, i111);
        }
        atomicAdd(p, i000 - bias);
        atomicAdd(p + 1, i100 - bias);
        atomicAdd(p + sx, i010 - bias);
        atomicAdd(p + sx + 1, i110 - bias);
        atomicAdd(p + sxy, i001 - bias);
        atomicAdd(p + sxy + 1, i101 - bias);
        atomicAdd(p + sxy + sx, i011 - bias);
        atomicAdd(p + sxy + sx + 1, i111 - bias);
        w *= inv_ratio;
        qx -= dx;
        qy -= dy;
        qz -= dz;
    }
}

// Cell bounds of a chunk's samples: the cell of its anchor (sample jh-1) and the cell the
// backward walk reaches at jl.
__device__ __forceinline__ void chunk_bounds(const Ray &R, const Anchor &an, int jl, int jh, int lo[3], int hi[3])
{
    const long long n = (long long)(jh - 1 - jl);
    const long long bx = an.x - n * R.d23x, by = an.y - n * R.d23y, bz = an.z - n * R.d23z;
    const int c0x = (int)(an.x >> 23), c0y = (int)(an.y >> 23), c0z = (int)(an.z >> 23);
    const int c1x = (int)(bx >> 23), c1y = (int)(by >> 23), c1z = (int)(bz >> 23);
    lo[0] = min(c0x, c1x); hi[0] = max(c0x, c1x) + 1;
    lo[1] = min(c0y, c1y); hi[1] = max(c0y, c1y) + 1;
    lo[2] = min(c0z, c1z); hi[2] = max(c0z, c1z) + 1;
}

// ---------------------------------------------------------------------------------
// the tiled traversal, adjoint (FWD = false) or forward (FWD = true)
// ---------------------------------------------------------------------------------
// Box extents stay below 256 voxels per axis (Q9.23 box-relative positions).
constexpr int kMaxBoxExtent = 255;

template <bool FWD, typename VT, typename PT>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm)
    tiled_kernel(const OpParams P, const VT *__restrict__ vol, PT *__restrict__ proj, float *__restrict__ acc,
                 uint32_t flags)
{
    extern __shared__ __align__(16) float box[];
    __shared__ int s_box[3][6];   // per chunk (rotating): min x,y,z and max x,y,z of the footprint
    __shared__ int s_rng[3][3];   // per aperture sample (rotating): first and last chunk, max |ray weight| bits

    // Grid: x = pixel-column tile, y = angle, z = pixel-row tile.  Blocks launch x fastest,
    // so the blocks resident at a time share one row tile -- one slab of z planes of the
    // volume and one band of the ray table, which then stay in L2 across the angles.
    // Lanes run down a pixel column (v), warps across columns (u): at every step the 32
    // samples of a warp are stacked along z, one voxel plane apart, so with an odd plane
    // stride their shared-memory words fall in distinct banks.
    const int tid = threadIdx.y * kTileV + threadIdx.x;
    const int u = blockIdx.x * kTileU + threadIdx.y;
    const int k = blockIdx.y;
    const int v = blockIdx.z * kTileV + threadIdx.x;
    const bool valid = u < P.nu && v < P.nv;

    float g = 0.f;
    if (FWD && valid) g = to_f(proj[((int64_t)k * P.nv + v) * P.nu + u]);
    if (tid < 18) s_box[tid / 6][tid % 6] = (tid % 6 < 3) ? INT_MAX : INT_MIN;
    if (tid < 9) s_rng[tid / 3][tid % 3] = (tid % 3 == 0) ? INT_MAX : (tid % 3 == 1) ? INT_MIN : 0;
    __syncthreads();

    const int pxy = P.px * P.py;
    float pix = 0.f;
    int n_chunk = 0;
    for (int a = 0; a < P.M; ++a) {
        const int ra = a % 3;
        Ray R;
        bool active = valid && (!FWD || g != 0.f);
        if (active)
            active = ray_begin(P, ((int64_t)a * P.nv + v) * P.nu + u, P.cs[k], R, !FWD && (flags & VAMRT_UNATTENUATED));
        int cf = INT_MAX, cl = INT_MIN;
        if (active) {
            cf = chunk_of(P, R, R.jlo);
            cl = (R.dy > kMinDy) ? chunk_of(P, R, R.jhi - 1) : cf;
            if (cl < cf) cl = cf;
        }
        const float wray = (FWD && active) ? g * R.w : 0.f;
        // the warp's shares are all non-negative: the subnormal conversion applies
        const bool nonneg = FWD && __all_sync(kFull, !(wray < 0.f));
        cf = __reduce_min_sync(kFull, cf);
        cl = __reduce_max_sync(kFull, cl);
        // |weights| >= 0 order like their bit patterns
        const int wbits = FWD ? __reduce_max_sync(kFull, __float_as_int(fabsf(wray))) : 0;
        if (threadIdx.x == 0 && cf <= cl) {
            atomicMin(&s_rng[ra][0], cf);
            atomicMax(&s_rng[ra][1], cl);
            if (FWD) atomicMax(&s_rng[ra][2], wbits);
        }
        __syncthreads();
        const int cmin = s_rng[ra][0], cmax = s_rng[ra][1];
        float scale = 0.f;
        if (FWD) {
            // fixed-point scale: a voxel takes at most cell_bound shares from each of the
            // block's rays, each at most max|w|; keep the block's sum below 2^31
            const float wmax = __int_as_float(s_rng[ra][2]);
            scale = fminf(2147483648.0f / (1.01f * (float)kThreads * P.cell_bound * wmax), 1e30f);
        }
        if (tid == 0) {
            s_rng[(a + 2) % 3][0] = INT_MAX;
            s_rng[(a + 2) % 3][1] = INT_MIN;
            s_rng[(a + 2) % 3][2] = 0;
        }
        float ray_acc = 0.f;

        // Chunks of kChunkVox voxels along y; a chunk whose box does not fit in shared memory
        // is retried as its two halves (block-uniform decision), and a half that still does
        // not fit runs on global memory.
        for (int c = cmin; c <= cmax; ++c) {
          int nsplit = 1;
          for (int part = 0; part < nsplit; ++part) {
            const int rb = n_chunk % 3;
            ++n_chunk;
            const int h0 = 2 * c + part * (2 / nsplit), h1 = h0 + 2 / nsplit;
            int jl = 0, jh = 0;
            if (active) range_samples(P, R, h0, h1, cmin, cmax, jl, jh);
            int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
            Anchor an{0, 0, 0};
            if (jl < jh) {
                an = anchor_at(R, jh);
                chunk_bounds(R, an, jl, jh, lo, hi);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lo[d] = __reduce_min_sync(kFull, lo[d]);
                hi[d] = __reduce_max_sync(kFull, hi[d]);
            }
            if (threadIdx.x == 0 && lo[0] != INT_MAX) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    atomicMin(&s_box[rb][d], lo[d]);
                    atomicMax(&s_box[rb][3 + d], hi[d]);
                }
            }
            __syncthreads();
            const int bx0 = s_box[rb][0] & ~3, by0 = s_box[rb][1], bz0 = s_box[rb][2];
            const int hx = s_box[rb][3], hy = s_box[rb][4], hz = s_box[rb][5];
            const bool lo_inside = s_box[rb][0] >= 0 && by0 >= 0 && bz0 >= 0;
            if (tid == 0) {
                const int nb = (rb + 2) % 3;
                s_box[nb][0] = s_box[nb][1] = s_box[nb][2] = INT_MAX;
                s_box[nb][3] = s_box[nb][4] = s_box[nb][5] = INT_MIN;
            }
            if (hx == INT_MIN) continue;                      // no samples in this range
            const int ex = ((hx + 4) & ~3) - bx0;             // x extent, a multiple of 4
            const int ey = hy + 1 - by0, ez = hz + 1 - bz0;
            const int sx = ex + 1, sxy = sx * (ey | 1);       // odd row and plane strides
            const int ex4 = ex >> 2;
            // the box path needs the box inside the padded grid (the backward walk's truncated
            // step can carry a sample a hair past a grid face: such ranges run on global
            // memory with exact positions) and extents a Q9.23 offset can hold
            const bool in_grid = lo_inside && hx <= P.px - 1 && hy <= P.py - 1 && hz <= P.pz - 1;
            const bool fits = (long long)sxy * ez <= kBoxFloats && ex <= kMaxBoxExtent && ey <= kMaxBoxExtent &&
                              ez <= kMaxBoxExtent;
            if (!fits && nsplit == 1 && in_grid) {
                nsplit = 2;          // the same decision in every thread: retry as two halves
                part = -1;
                continue;
            }
            if (fits && in_grid) {
                const SlotWalk sw(ex4, ey);
                if (!FWD) {
                    const int64_t gstep = (int64_t)sw.phases * pxy;
                    const int bstep = sw.phases * sxy;
                    for (int it = tid; it < sw.items; it += kThreads) {
                        int zp, yy, x4;
                        sw.at(it, ex4, zp, yy, x4);
                        const VT *src = vol + ((int64_t)(bz0 + zp) * pxy + (int64_t)(by0 + yy) * P.px + bx0 + 4 * x4);
                        float *b = box + zp * sxy + yy * sx + 4 * x4;
                        // unrolled so that several planes' loads are in flight before their stores
#pragma unroll 2
                        for (int zz = zp; zz < ez; zz += sw.phases) {
                            const float4 q = ld4(src);
                            b[0] = q.x; b[1] = q.y; b[2] = q.z; b[3] = q.w;
                            src += gstep;
                            b += bstep;
                        }
                    }
                } else {
                    // the box base is 16-byte aligned and kBoxFloats a multiple of 4
                    float4 *b4 = reinterpret_cast<float4 *>(box);
                    const int n = (sxy * ez + 3) >> 2;
                    for (int i = tid; i < n; i += kThreads) b4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncthreads();
                if (jl < jh) {
                    if (!FWD)
                        ray_acc += exp2f(R.att * ((float)jl + 0.5f)) *
                                   walk_gather_box(R, an, jl, jh, bx0, by0, bz0, box, sx, sxy);
                    else if (nonneg)
                        walk_scatter_box<true>(R, an, jl, jh, wray, scale, bx0, by0, bz0,
                                               reinterpret_cast<int *>(box), sx, sxy);
                    else
                        walk_scatter_box<false>(R, an, jl, jh, wray, scale, bx0, by0, bz0,
                                                reinterpret_cast<int *>(box), sx, sxy);
                }
                if (FWD) {
                    __syncthreads();
                    const float inv = 1.0f / scale;
                    const int *ib = reinterpret_cast<const int *>(box);
                    const int64_t gstep = (int64_t)sw.phases * pxy;
                    const int bstep = sw.phases * sxy;
                    for (int it = tid; it < sw.items; it += kThreads) {
                        int zp, yy, x4;
                        sw.at(it, ex4, zp, yy, x4);
                        float *g = acc + ((int64_t)(bz0 + zp) * pxy + (int64_t)(by0 + yy) * P.px + bx0 + 4 * x4);
                        const int *b = ib + zp * sxy + yy * sx + 4 * x4;
                        for (int zz = zp; zz < ez; zz += sw.phases) {
                            const int b0 = b[0], b1 = b[1], b2 = b[2], b3 = b[3];
                            if ((b0 | b1 | b2 | b3) != 0)
                                red_v4(g, make_float4((float)b0 * inv, (float)b1 * inv, (float)b2 * inv, (float)b3 * inv));
                            g += gstep;
                            b += bstep;
                        }
                    }
                }
            } else if (jl < jh) {
                if (!FWD)
                    ray_acc += walk_gather_global(P, R, jl, jh, vol);
                else
                    walk_scatter_global(P, R, jl, jh, wray, acc);
            }
          }
        }
        if (!FWD && active) pix = fmaf(R.w, ray_acc, pix);
    }
    if (!FWD && valid) {
        PT *out = proj + (((int64_t)k * P.nv + v) * P.nu + u);
        if (flags & VAMRT_ACCUMULATE) pix += to_f(*out);
        if (flags & VAMRT_CLAMP_NONNEG) pix = fmaxf(pix, 0.f);
        st_val(out, pix);
    }
}

inline unsigned grid_for(const vamrt_projector *p, int64_t n, int threads)
{
    int64_t want = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)p->num_sms * 16;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (unsigned)want;
}

inline dim3 op_grid(const OpParams &P)
{
    return dim3((P.nu + kTileU - 1) / kTileU, P.n_angles, (P.nv + kTileV - 1) / kTileV);
}

constexpr size_t kSmem = sizeof(float) * kBoxFloats;

template <bool FWD, typename VT, typename PT>
cudaError_t launch_tiled(const OpParams &P, const VT *vol, PT *proj, float *acc, uint32_t flags, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(tiled_kernel<FWD, VT, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e != cudaSuccess) return e;
    tiled_kernel<FWD, VT, PT><<<op_grid(P), dim3(kTileV, kTileU), kSmem, s>>>(P, vol, proj, acc, flags);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

// Storage types: FP32, BF16 or FP16 (every sum is FP32 whatever the storage).
template <typename F>
cudaError_t with_storage(vamrt_dtype dt, void *ptr, F &&f)
{
    if (dt == VAMRT_F32) return f((float *)ptr);
    if (dt == VAMRT_BF16) return f((__nv_bfloat16 *)ptr);
    return f((__half *)ptr);
}

cudaError_t launch_pad(const vamrt_projector *p, const void *vol, vamrt_dtype dt, cudaStream_t s)
{
    const OpParams &P = p->op;
    const unsigned grid = grid_for(p, p->pad_elems, 256);
    return with_storage(dt, const_cast<void *>(vol), [&](auto *v) {
        using VT = std::remove_pointer_t<decltype(v)>;
        pad_kernel<VT><<<grid, 256, 0, s>>>(v, (VT *)p->scratch, P.nx, P.ny, P.nz, P.px, P.py, p->pad_elems);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_adjoint(const vamrt_projector *p, vamrt_dtype vol_dt, void *proj, vamrt_dtype proj_dt,
                           uint32_t flags, cudaStream_t s)
{
    const OpParams &P = p->op;
    return with_storage(vol_dt, p->scratch, [&](auto *vol) {
        return with_storage(proj_dt, proj, [&](auto *pr) {
            return launch_tiled<false>(P, (const std::remove_pointer_t<decltype(vol)> *)vol, pr, nullptr, flags, s);
        });
    });
}

cudaError_t launch_forward_acc(const vamrt_projector *p, const void *proj, vamrt_dtype proj_dt, float *acc,
                               cudaStream_t s)
{
    const OpParams &P = p->op;
    const float *none = nullptr;
    return with_storage(proj_dt, const_cast<void *>(proj),
                        [&](auto *pr) { return launch_tiled<true>(P, none, pr, acc, 0u, s); });
}

cudaError_t launch_forward(const vamrt_projector *p, const void *proj, vamrt_dtype proj_dt, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p->scratch, 0, sizeof(float) * p->pad_elems, s);
    if (e != cudaSuccess) return e;
    return launch_forward_acc(p, proj, proj_dt, p->scratch, s);
}

cudaError_t launch_unpad_acc(const vamrt_projector *p, const float *acc, void *dose, vamrt_dtype dt, uint32_t flags,
                             cudaStream_t s)
{
    const OpParams &P = p->op;
    const unsigned grid = grid_for(p, (int64_t)P.nx * P.ny * P.nz, 256);
    const int accumulate = (flags & VAMRT_ACCUMULATE) ? 1 : 0;
    return with_storage(dt, dose, [&](auto *d) {
        using DT = std::remove_pointer_t<decltype(d)>;
        unpad_kernel<DT><<<grid, 256, 0, s>>>(acc, d, P.nx, P.ny, P.nz, P.px, P.py, accumulate);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_unpad(const vamrt_projector *p, void *dose, vamrt_dtype dt, uint32_t flags, cudaStream_t s)
{
    return launch_unpad_acc(p, p->scratch, dose, dt, flags, s);
}

}  // namespace vamrt
