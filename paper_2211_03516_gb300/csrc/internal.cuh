// Internal declarations shared by the vamrt CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "../../include/vamrt.h"

namespace vamrt {

// Largest optimiser run whose error history the handle keeps on the device.
constexpr int kMaxHistory = 4096;
// Partial-sum slots for the deterministic two-pass reductions.
constexpr int kRedBlocks = 1024;

// Operator tiling: a block owns kTileU x kTileV pixels of one angle and walks their rays
// chunk by chunk along the projection axis (kChunkVox voxels of the theta = 0 frame's y
// per chunk).  Each chunk's voxel footprint is staged in a shared-memory box of at most
// kBoxFloats floats; a chunk whose box would not fit runs straight on global memory.
constexpr int kTileU = 8;
constexpr int kTileV = 32;
constexpr int kThreads = kTileU * kTileV;
constexpr int kChunkVox = 20;
constexpr int kBoxFloats = 18 * 1024;
constexpr int kBlocksPerSm = 3;

// Per-launch constants of the two operators.  Positions are in padded index
// coordinates: the scratch volume has a zero halo of one voxel on every face (and its
// rows are padded to a multiple of 4 floats), so voxel (i,j,k) of the caller's grid
// sits at (i+1, j+1, k+1).
struct OpParams {
    const double4_32a *A; // (e_x, e_y, e_z, delta) in voxels, theta = 0 frame, relative to the axis
    const double4_32a *B; // (d_x, d_y, d_z, T1 T2 delta_mm / M)
    const int2 *J;        // [j_lo, j_hi) samples whose footprint reaches the grid
    const double2 *cs;    // (cos theta_k, sin theta_k), FP64
    int nu, nv, M, n_angles;
    int nx, ny, nz;       // caller's grid
    int px, py, pz;       // padded extents (px a multiple of 4)
    double cx, cy, cz;    // axis position in padded index coordinates
    float neg_mu_vox_log2e;  // -mu h log2(e): attenuation = exp2(this * s_vox)
    float y0;             // start of chunk 0 on the theta = 0 frame's y axis, voxels
    float cell_bound;     // most samples of one ray whose footprint holds a given voxel
    float h_over_m;       // voxel pitch (mm) / rays per pixel: delta_mm / M = delta_vox * h_over_m
};

// Per-ray constants of the FP64 tracer.
struct TraceParams {
    const double *pupil_xy;   // device, M pairs (aperture = VAMRT_APERTURE_LIST)
    int aperture;             // VAMRT_APERTURE_*
    int per_pixel;            // jitter drawn per pixel
    unsigned long long seed;
    int strat_n;              // strata per side (stratified aperture)
    int nu, nv, M, nz;
    double pu, pv;
    double pupil_mm, f_number;
    int telecentric, chief_only;
    double r_in, r_out, n_out, n_glass, n_resin;
    double h, ds;
    const double *surf;       // device, n_surf x (y, radius, n_after, clear, stop flag); n_surf = 0: pupil model
    int n_surf;
    double obj_y, mag, aim, stop_r;
};

}  // namespace vamrt

struct vamrt_projector {
    vamrt_geometry g;          // copy; host pointers cleared
    int device;
    int num_sms;
    int64_t n_rays;
    int64_t rays_in_resin;
    uint64_t samples_per_angle;
    uint64_t device_bytes;
    double4_32a *tabA;         // FP64: a large grid's positions need more than FP32's 24 bits
    double4_32a *tabB;
    int2 *tabJ;
    double2 *cs;
    float *scratch;            // padded FP32 volume, pad_elems floats
    int64_t pad_elems;
    double *red;               // kRedBlocks partials + scalars
    double *hist;              // kMaxHistory errors
    float *dmax;               // one float, max of the dose
    double *host_err;          // pinned, 4 doubles: the optimiser's E and VER counts
    vamrt::OpParams op;
};

namespace vamrt {

// Count of kernel launches issued by the library (vamrt_launch_count).
void count_launches(unsigned n);
// Set the calling thread's vamrt_last_error() text.
void set_error(const char *msg);

// raytable.cu
cudaError_t launch_raytable(const TraceParams &T, double4_32a *A, double4_32a *B, int2 *J,
                            unsigned long long *counters, cudaStream_t s);

// static_dose.cu: device address of the allocation-free dose entry point's static
// accumulator on the current device `dev` (loads its module on first use)
cudaError_t static_acc_address(int dev, float **out);

// operators.cu
cudaError_t operators_init();
cudaError_t launch_pad(const vamrt_projector *p, const void *vol, vamrt_dtype dt, cudaStream_t s);
cudaError_t launch_adjoint(const vamrt_projector *p, vamrt_dtype vol_dt, void *proj, vamrt_dtype proj_dt,
                           uint32_t flags, cudaStream_t s);
cudaError_t launch_forward(const vamrt_projector *p, const void *proj, vamrt_dtype proj_dt, cudaStream_t s);
cudaError_t launch_unpad(const vamrt_projector *p, void *dose, vamrt_dtype dt, uint32_t flags, cudaStream_t s);
// The same two steps on a caller-chosen FP32 accumulator of p->pad_elems floats (the
// caller zeroes it first).
cudaError_t launch_forward_acc(const vamrt_projector *p, const void *proj, vamrt_dtype proj_dt, float *acc,
                               cudaStream_t s);
cudaError_t launch_unpad_acc(const vamrt_projector *p, const float *acc, void *dose, vamrt_dtype dt, uint32_t flags,
                             cudaStream_t s);

// loss.cu: loss3 = device doubles {L, 1/|P|, 1/|Q|}; grad may be NULL
cudaError_t launch_threshold_loss(const vamrt_projector *p, const void *dose, vamrt_dtype dose_dt,
                                  const float *target, float d_l, float d_h, double *loss3, void *grad,
                                  vamrt_dtype grad_dt, cudaStream_t s);

// loss.cu: out2 = device {count, sum} of x over target > 1/2 (target given) or over x > 0
// (target NULL), summed in a fixed order
cudaError_t launch_masked_sum(const vamrt_projector *p, const void *x, vamrt_dtype dt, const float *target,
                              int64_t n, double *out2, cudaStream_t s);
// loss.cu: master = sc * x in FP32; x (in dt) rewritten from master when it is not master itself
cudaError_t launch_scale_master(const vamrt_projector *p, void *x, vamrt_dtype dt, float *master, int64_t n, float sc,
                                cudaStream_t s);

// ver.cu: out3 = device {best mismatch count, best threshold index, resin voxels}
cudaError_t launch_ver(const vamrt_projector *p, const void *dose, vamrt_dtype dt, const float *target,
                       long long *out3, cudaStream_t s);

// ramlak.cu (Radon-method baseline): rows x nu floats, in place allowed
cudaError_t launch_ramlak(const float *in, float *out, int64_t rows, int nu, double pixel_mm, int clamp,
                          cudaStream_t s);

// conv3d_tc.cu (tensor-core convolution of the warm-start network)
cudaError_t launch_conv3d_tc(const void *X, const void *Wt, const float *bias, void *Y, int out_f32, int D, int H,
                             int W, int Cin, int Cout, int taps, int relu, int *err, cudaStream_t s);

// conv3d_wgrad.cu: plan of the TMA-fed weight gradient (host only; false for shapes it
// cannot take)
struct WgradPlan {
    int Mtot, nmt, tpg, kp, KS, BX, nstage, cwA, cwB, slots, slot_bytes, per_sm, ncols, ngroups, nsplit, spb;
};
bool plan_wgrad_tma(int D, int H, int W, int Cin, int Cout, int taps, int sms, WgradPlan *pl);

// conv3d_wgrad.cu: the driver's tensor-map encoder (cuTensorMapEncodeTiled, through the
// runtime's driver entry point); NULL when the driver does not provide it
PFN_cuTensorMapEncodeTiled_v12000 tma_encoder();

// conv3d_halo.cu (persistent halo-tile variant; W % 8 == 0).  launch returns
// cudaErrorNotSupported for shapes it does not take.
struct ConvHaloPlan {
    int TZ, TY, Nt, T, WP, PT, NX, rowtile, mg, adv, a_bytes, box_bytes, stage_bytes, ncols, ry, nslice, nitems;
};
bool plan_conv3d_halo(int D, int H, int W, int Cin, int Cout, int taps, int sms, ConvHaloPlan *pl);
cudaError_t launch_conv3d_halo(const void *X, const void *Wt, const float *bias, void *Y, int out_f32, int D, int H,
                               int W, int Cin, int Cout, int taps, int relu, int *err, cudaStream_t s);

cudaError_t launch_conv3d_wgrad_tc(const void *X, const void *dY, float *dW, int D, int H, int W, int Cin, int Cout,
                                   int taps, int *err, cudaStream_t s);

// nn_ops.cu
cudaError_t nn_resample(int op, const void *in, void *out, int D, int H, int W, int C, cudaStream_t s);
cudaError_t nn_concat(const void *a, int ca, const void *b, int cb, void *out, int64_t npos, int backward,
                      cudaStream_t s);
cudaError_t nn_relu_bwd(const void *y, void *dy, int64_t n, cudaStream_t s);
cudaError_t nn_bias_grad(const void *dy, float *db, int64_t npos, int C, cudaStream_t s);
cudaError_t nn_flip_weights(const void *w, void *wt, int cout, int taps, int cin, cudaStream_t s);
cudaError_t nn_adam(float *p, const float *g, float *m, float *v, void *pb, int64_t n, float lr, float b1, float b2,
                    float eps, int step, bool nonneg, cudaStream_t s);
cudaError_t nn_prepare_input(const float *proj, void *x, int A, int V, int U, int Dp, float scale, cudaStream_t s);
cudaError_t nn_head_mse(const float *z, int cz, const float *base, float in_scale, const float *target,
                        float target_scale, float *out, float out_scale, void *dz, int A, int V, int U, int Dp,
                        double *loss, cudaStream_t s);
cudaError_t nn_add(const void *x, void *y, int64_t n, cudaStream_t s);
cudaError_t nn_projected_step(float *g, const float *grad, float eta, int64_t n, cudaStream_t s);
cudaError_t nn_absmax(const float *x, int64_t n, float *out, cudaStream_t s);

// export.cu (8-bit export of projections, Sec. 2.7)
cudaError_t launch_export_u8(const vamrt_projector *p, const void *proj, vamrt_dtype dt, unsigned char *codes,
                             float *dequant, double *clip, cudaStream_t s);

// osmo.cu
cudaError_t launch_sum(const vamrt_projector *p, const float *x, double *out, cudaStream_t s);
cudaError_t launch_osmo_step(const vamrt_projector *p, const float *target, float *model, void *dose,
                             vamrt_dtype dose_dt, const double *fsum, double *err_out, int residual, float alpha,
                             float mu, float *prev, cudaStream_t s);

}  // namespace vamrt
