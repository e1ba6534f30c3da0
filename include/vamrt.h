/*
 * vamrt — GB300-native 3D ray-traced projection and dose operators for tomographic
 * volumetric additive manufacturing (Webber et al., "Versatile volumetric additive
 * manufacturing with 3D ray tracing", arXiv 2211.03516).
 *
 * C ABI.  Every entry point takes plain pointers and sizes, returns a vamrt_status and
 * never lets an exception or exit() cross the boundary.  Device buffers are owned by
 * the caller unless stated otherwise; the library owns only a projector handle (its ray
 * table, angle table and one scratch volume) and small reduction buffers.
 *
 * Conventions (shared by every call):
 *   - Volume layout [nz][ny][nx], x fastest; voxel (i,j,k) has its centre at
 *     ((i-(nx-1)/2) h, (j-(ny-1)/2) h, (k-(nz-1)/2) h) in the vial frame; z is the vial
 *     (rotation) axis.  Values outside the grid count as zero.
 *   - Projection layout [n_angles][nv][nu], u fastest; pixel (u,v) images to the point
 *     ((u-(nu-1)/2) pu, 0, (v-(nv-1)/2) pv) of the best-focus plane y = 0, which contains
 *     the rotation axis (Sec. 2.8).  Light travels +y.
 *   - At angle theta_k a point x of the fixed (projector) frame sits at R_z(theta_k) x
 *     in the vial frame, R_z(t) = [[cos t, -sin t], [sin t, cos t]].
 *   - Calls are stream-ordered and asynchronous unless stated.  A projector may be used
 *     by one stream at a time (its scratch volume is shared by the operators).
 *   - On error the outputs are unspecified but no access outside the caller's buffers
 *     happens; vamrt_last_error() gives a one-line reason for the calling thread.
 */
#ifndef VAMRT_H
#define VAMRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VAMRT_OK = 0,
    VAMRT_EINVAL = 1,          /* an argument is out of range, NULL or inconsistent */
    VAMRT_EUNSUPPORTED = 2,    /* a valid request this library does not implement */
    VAMRT_ECUDA = 3,           /* a CUDA runtime call failed (message in vamrt_last_error) */
    VAMRT_ENOMEM = 4,          /* device allocation failed */
    VAMRT_NOT_CONVERGED = 5,   /* the optimiser hit its iteration cap above tolerance */
    VAMRT_NUMERIC = 6          /* NaN/Inf or an all-zero dose met in a reduction */
} vamrt_status;

typedef enum {
    VAMRT_F32 = 0,             /* float */
    VAMRT_BF16 = 1,            /* bfloat16 storage; all sums are FP32 */
    VAMRT_F16 = 2              /* IEEE binary16 storage; all sums are FP32.  Values beyond 65504
                                  in magnitude round to infinity: scale inputs to its range */
} vamrt_dtype;

/* Operator flags */
#define VAMRT_ACCUMULATE   1u  /* add into the output instead of overwriting it */
#define VAMRT_CLAMP_NONNEG 2u  /* adjoint only: write max(0, result) (OSMO's clamp, Sec. 2.7) */
#define VAMRT_UNATTENUATED 4u  /* adjoint only: the paper-literal projection of Sec. 2.4, the sum of
                                  the (trilinear-weighted) voxels each ray crosses: weight
                                  delta / M per sample, no Fresnel or Beer-Lambert factor (no
                                  longer the transpose of the dose operator) */

/*
 * Printer, vial and grid description (Sec. 2.1, 2.5, 2.6).  All lengths in mm.
 *   pupil_mm    distance from the rotation axis to the aperture stop, which sits on the
 *               -y side.  INFINITY selects a telecentric projector.  Non-telecentric:
 *               ray a of pixel (u,v) leaves the stop point (xi_a D/2, -pupil_mm, eta_a D/2),
 *               D = pupil_mm / f_number, and passes through the pixel's image point.
 *               Telecentric: the ray crosses the image point with direction proportional
 *               to (-xi_a t, 1, -eta_a t), t = 1/(2 f_number).
 *   f_number    INFINITY = zero etendue (all rays of a pixel are its chief ray).
 *   aperture    how the rays_per_pixel stop points (xi, eta) in the unit disk are chosen
 *               (Sec. 2.1: a pixel's rays leave points of the aperture stop, the chief ray
 *               its centre; the paper fills the stop hexagonally):
 *                 VAMRT_APERTURE_LIST        the HOST array pupil_xy (copied; NULL = one chief ray),
 *                 VAMRT_APERTURE_CHIEF       one ray, (0, 0),
 *                 VAMRT_APERTURE_STRATIFIED  rays_per_pixel = n^2: ray a = i n + k takes the point
 *                                            (2 (i + J0)/n - 1, 2 (k + J1)/n - 1) of stratum (i, k)
 *                                            of [-1,1]^2, mapped to the disk by Shirley and
 *                                            Chiu's concentric map,
 *                 VAMRT_APERTURE_SUNFLOWER   r = sqrt((a + 1/2)/M), azimuth a g + 2 pi J,
 *                                            g = pi (3 - sqrt 5) the golden angle, J = J0 of a = 0,
 *                 VAMRT_APERTURE_HEX         13 rays: the points of a hexagonal lattice of spacing
 *                                            1/2 inside the disk (centre; 6 at r = 1/2, azimuths
 *                                            0, 60, .. 300 degrees; 6 at r = sqrt(3)/2, 30, 90, ..
 *                                            330 degrees).
 *               Jitter numbers Jc (c = 0, 1) of ray a of pixel (u, v): the top 53 bits of
 *               splitmix64(seed ^ (u + 2^20 v + 2^40 a + 2^56 c)) times 2^-53, with u = v = 0
 *               unless aperture_flags has VAMRT_JITTER_PER_PIXEL (splitmix64: the Weyl step
 *               0x9E3779B97F4A7C15 then the mix of Steele, Lea and Flood / Vigna).
 *   vial        inner radius r_inner_mm, glass wall wall_mm, refractive indices outside,
 *               glass, resin; Fresnel losses (unpolarised) at the outer and inner surface;
 *               tracing stops at the inner wall on the far side (Sec. 2.1).
 *   mu_per_mm   Beer-Lambert absorption coefficient of the resin (Sec. 2.5).
 *   angles_rad  HOST array of n_angles angles, copied; NULL = 2 pi k / n_angles.
 *   step_vox    nominal spacing of the samples on a ray, in voxels (0 = 0.5, the 2x
 *               super-sampling of Sec. 2.2).  Each in-resin segment of length ell gets
 *               K = ceil(ell / (step_vox h) - 1e-9) midpoint samples s_j = (j+1/2) ell/K.
 *   n_surfaces  0: the ideal-pupil model above.  > 0: a lens train of n_surfaces surfaces
 *               (HOST array `surfaces`, copied) between the pixel array and the vial
 *               replaces it (Sec. 2.1: rays refract at every optical element; Sec. 2.6.2:
 *               the telecentric printer's lenses and iris).  Pixel (u,v) then sits at
 *               Q_uv / magnification in the plane y = object_y_mm (Q_uv its image point in
 *               y = 0); aperture sample (xi, eta) leaves it with direction proportional to
 *               (xi r_s / aim_mm, 1, eta r_s / aim_mm), r_s = the stop's clear_mm (an
 *               object-space telecentric launch aimed paraxially at the stop; for a
 *               telecentric relay aim_mm is the focal length before the stop).  At each
 *               surface the ray refracts by the vector Snell law (transmission 1: coated
 *               lenses) and is blocked outside the clear aperture; blocked rays carry no
 *               light.  pupil_mm and f_number are then ignored.
 * The grid must enclose the resin cylinder: r_inner_mm / voxel_mm <= (min(nx,ny)+1)/2 - 0.01.
 */
#define VAMRT_APERTURE_LIST 0
#define VAMRT_APERTURE_CHIEF 1
#define VAMRT_APERTURE_STRATIFIED 2
#define VAMRT_APERTURE_SUNFLOWER 3
#define VAMRT_APERTURE_HEX 4
#define VAMRT_JITTER_PER_PIXEL 1u  /* aperture_flags: jitter drawn per pixel, not shared by all */

typedef struct {
    double y_mm;               /* vertex on the optical axis (the y axis through x = z = 0) */
    double radius_mm;          /* radius of curvature, centre at y_mm + radius_mm; INFINITY = plane */
    double n_after;            /* index behind the surface (in front: the previous surface's, or n_outside) */
    double clear_mm;           /* clear semi-aperture (the stop: its radius) */
    int32_t is_stop;           /* nonzero: the aperture stop, a plane that blocks and does not refract */
} vamrt_surface;

typedef struct {
    int32_t nx, ny, nz;
    double voxel_mm;
    int32_t nu, nv;
    double pixel_u_mm, pixel_v_mm;
    double pupil_mm;
    double f_number;
    int32_t rays_per_pixel;
    const double *pupil_xy;
    double r_inner_mm, wall_mm;
    double n_outside, n_glass, n_resin;
    double mu_per_mm;
    int32_t n_angles;
    const double *angles_rad;
    double step_vox;
    int32_t n_surfaces;              /* 0 = ideal pupil; 1..64 = lens train (see above) */
    const vamrt_surface *surfaces;   /* HOST array in increasing y_mm, exactly one stop, last n_after = n_outside */
    double object_y_mm;              /* pixel array plane, before the first surface */
    double magnification;            /* paraxial image / object height (nonzero) */
    double aim_mm;                   /* launch aim distance (> 0) */
    int32_t aperture;                /* VAMRT_APERTURE_* (0 = LIST: pupil_xy) */
    uint32_t aperture_flags;         /* VAMRT_JITTER_PER_PIXEL */
    uint64_t seed;                   /* jitter seed */
} vamrt_geometry;

typedef struct vamrt_projector vamrt_projector;   /* opaque */

typedef struct {
    int64_t n_rays;            /* nu * nv * rays_per_pixel */
    int64_t rays_in_resin;     /* rays that reach the resin */
    uint64_t samples_per_pass; /* n_angles * sum over rays of samples reaching the grid */
    uint64_t scratch_bytes;    /* device bytes owned by the handle (table + scratch) */
} vamrt_info;

/*
 * Build a projector: validates the geometry on the host, then traces every
 * (pixel, aperture-sample) ray through the vial once, in FP64 on the device (Sec. 2.1:
 * ray generation, vector Snell's law and Fresnel transmission at both cylinder surfaces,
 * the in-resin segment).  The vial is rotationally symmetric about z, so the segment at
 * angle theta_k is the theta = 0 segment rotated; only the theta = 0 table is stored
 * (72 B per ray, FP64 positions and directions).  Synchronises `stream` (a cudaStream_t, NULL = legacy default)
 * before returning.  *out receives a handle to release with vamrt_destroy_projector.
 * Errors: EINVAL (bad geometry), ENOMEM, ECUDA.
 */
vamrt_status vamrt_make_projector(const vamrt_geometry *geom, void *stream, vamrt_projector **out);

/* Release a projector and its device memory (synchronises the device first). NULL is a no-op. */
void vamrt_destroy_projector(vamrt_projector *p);

/* Sizes, ray counts and the exact number of ray-voxel samples one operator pass visits. */
vamrt_status vamrt_get_info(const vamrt_projector *p, vamrt_info *info);

/* Samples per pass (same as vamrt_get_info's samples_per_pass). */
vamrt_status vamrt_sample_count(const vamrt_projector *p, uint64_t *samples_per_pass);

/*
 * Projection operator, the adjoint A^T (Sec. 2.4, with Sec. 2.5's transmission factors):
 *   proj[k][v][u] = sum_a sum_j c_j sum_{8 corners} w_c vol[c],
 *   c_j = (T1 T2 / M) exp(-mu s_j) delta,  w_c = trilinear weight (Sec. 2.2).
 * vol: device [nz][ny][nx] of vol_dtype; proj: device [n_angles][nv][nu] of proj_dtype.
 * flags: VAMRT_ACCUMULATE, VAMRT_CLAMP_NONNEG, VAMRT_UNATTENUATED.  Uses the handle's scratch volume.
 * Errors: EINVAL (NULL pointers, unknown dtype/flags), ECUDA.
 */
vamrt_status vamrt_adjoint(vamrt_projector *p, const void *vol, vamrt_dtype vol_dtype,
                           void *proj, vamrt_dtype proj_dtype, uint32_t flags, void *stream);

/*
 * Dose operator A (Sec. 2.5): every sample of every ray adds
 *   proj[k][v][u] * c_j * w_c
 * to each of its 8 trilinear corner voxels, over all angles; A is exactly the transpose
 * of vamrt_adjoint.  Sums run in an FP32 scratch volume owned by the handle (summation
 * order is not deterministic); dose gets the result in dose_dtype.
 * flags: VAMRT_ACCUMULATE.  Errors: EINVAL, ECUDA.
 */
vamrt_status vamrt_forward_dose(vamrt_projector *p, const void *proj, vamrt_dtype proj_dtype,
                                void *dose, vamrt_dtype dose_dtype, uint32_t flags, void *stream);

/*
 * Dose operator with no device allocation: the same computation and arguments as
 * vamrt_forward_dose, but the FP32 accumulator is a fixed, statically allocated device
 * array of 4,194,304 floats (16 MiB) instead of the projector's scratch volume.  The
 * paper has no counterpart; this entry point exists for callers that cannot allocate
 * device memory (memory owned by another allocator or budgeted up front, or code that
 * must not allocate where it calls).  The call itself makes no cudaMalloc, cudaFree or
 * other allocating call; the projector (made earlier) supplies the ray table.
 *   - Limit: the padded grid, (nx+2 rounded up to a multiple of 4) x (ny+2) x (nz+2),
 *     must be at most 4,194,304 voxels (e.g. 158^3); larger grids return EINVAL.
 *   - The array exists once per device for the life of the process (every device that
 *     loads the library holds the 16 MiB) and is shared by all calls and projectors: each
 *     call first clears the part it uses, and calls that overlap on the GPU (other streams,
 *     other threads) race on it.  Serialise them.
 *   - The library's device code loads lazily: the array is created on a device, and its
 *     device address looked up, when vamrt_make_projector runs there (that call allocates
 *     anyway), so the projector's own device already holds it and this call only reads
 *     the cached address.  After a device reset (a new context) the first call looks the
 *     address up again, which loads the array anew (16 MiB): make that call before any
 *     CUDA stream capture, or make a new projector first.
 *   - The current device must be the projector's device.
 * Errors: EINVAL (NULL, dtype other than F32 / BF16, flags, grid too large, wrong device), ECUDA.
 */
vamrt_status vamrt_forward_dose_static(const vamrt_projector *p, const void *proj, vamrt_dtype proj_dtype,
                                       void *dose, vamrt_dtype dose_dtype, uint32_t flags, void *stream);

/*
 * Projection optimisation (Sec. 2.7).  The paper runs the object-space model
 * optimisation of Rackson et al. with both operators replaced by the ray-traced ones
 * and stops once the absolute relative error between target and simulated dose is below
 * 0.5 %.  Iteration, per the reading this library implements:
 *   g = max(0, A^T m);  d = A g;  dn = d / max_resin(d);
 *   E = sum |dn - f| / sum f;  V = voxel error rate of dn (vamrt_voxel_error_rate);
 *   m <- max(0, m + beta (f - dn) + mu (m - m_prev));
 *   stop once V < tol (params.stop = VAMRT_STOP_VER, the default) or E < tol
 *   (VAMRT_STOP_ERROR),
 * max_resin the maximum over the resin voxels (centres within r_inner_mm of the axis).
 * The paper's "absolute relative error" is read as V: the target against the dose as it
 * prints (thresholded), relative to the resin volume.  E, the dose's L1 error, cannot
 * fall to 0.5 % for a binary target (the dose is never zero in the void along rays that
 * cross the part) and is reported beside it.
 * beta = 1, mu = 0 is the plain update (params.step, 0 also meaning 1; params.momentum).
 * beta > 1 over-relaxes the model update and mu > 0 adds heavy-ball momentum -- neither is
 * in the paper; beta = 4, mu = 0.5 reaches the plain loop's final voxel error rate in 10 of
 * 30 iterations on the 256^3 test workload (13 without momentum).  With mu > 0 the
 * previous model lives in prev_model (in: the model before the one passed in -- a copy of
 * it to start at rest; out: updated), so a loop of single-iteration calls keeps its
 * momentum.
 * target: device f32 [nz][ny][nx] (the binary part f).  model: device f32, in = m0
 * (copy the target there for OSMO's start), out = the updated model.  proj: device
 * [n_angles][nv][nu] in proj_dtype, out = g of the last iteration.  dose: device
 * [nz][ny][nx] in dose_dtype, out = dn of the last iteration.
 * Synchronises `stream` once every check_every iterations to read E and V (V is computed
 * on those iterations only).
 */
typedef struct {
    int32_t max_iter;          /* 1 .. 4096 */
    double tol;                /* stop once E < tol (0.005 in the paper) */
    int32_t check_every;       /* read E on the host every this many iterations (>= 1) */
    vamrt_dtype proj_dtype;    /* storage of g */
    vamrt_dtype dose_dtype;    /* storage of dn */
    int32_t timing;            /* nonzero: time each phase with CUDA events on `stream` */
    int32_t mode;              /* VAMRT_OPT_OBJECT (the reading above), VAMRT_OPT_PROJECTIONS or VAMRT_OPT_GRADIENT */
    double step;               /* object mode: beta in [0, 64] (0 = 1); projection mode: alpha in (0, 1];
                                  gradient mode: Adam step factor in (0, 16] (0 = 0.8) */
    double momentum;           /* object mode: mu in [0, 1) (0 = none) */
    float *prev_model;         /* device f32 [nz][ny][nx], required when momentum > 0; see above */
    int32_t stop;              /* VAMRT_STOP_VER (0) or VAMRT_STOP_ERROR */
    double d_l, d_h;           /* gradient mode: the loss thresholds (both 0 = 0.8 and 1.0) */
} vamrt_opt_params;

#define VAMRT_STOP_VER 0
#define VAMRT_STOP_ERROR 1

/* Optimiser modes.  VAMRT_OPT_OBJECT iterates on the model m (model in = m0).
 * VAMRT_OPT_PROJECTIONS iterates on the projections themselves, starting from proj (in =
 * g0, e.g. a learned warm start): d = A g; dn = d / max(d); E as above;
 * g <- max(0, g + alpha A^T (f - dn)) -- with alpha = 1 the update OSMO makes to g = A^T m
 * when the model clamp is inactive; the model buffer is the residual workspace
 * (out = alpha (f - dn)). */
#define VAMRT_OPT_OBJECT 0
#define VAMRT_OPT_PROJECTIONS 1
/* VAMRT_OPT_GRADIENT: the differentiable path (not in the paper) -- projected Adam steps
 * on the thresholded dose loss of vamrt_threshold_loss, starting from proj (in = g0 >= 0,
 * e.g. a learned warm start; proj_dtype F32 or BF16, else EUNSUPPORTED).  g0 is first
 * scaled so that the part's mean dose is 1 (the thresholds' scale), then per iteration
 *   D = A g (stored in dose_dtype);  L, dL/dD (FP32, in the model buffer: volume workspace);
 *   grad = A^T dL/dD;  Adam step on an FP32 master copy of g (step size params.step x the
 *   mean positive projection after scaling, 0 = 0.8; moments 0.9 / 0.999), g >= 0;
 * E = L; V = the voxel error rate of D, each read every check_every iterations and
 * compared with tol as above.  Out: proj = g after the last step, dose = D of the last
 * iteration (before its step).  Allocates its FP32 state (3 or 4 projection-sized arrays)
 * for the call.  adjoint_ms times the gradient's projection, forward_ms the doses (and the
 * scaling), update_ms the loss and the Adam steps. */
#define VAMRT_OPT_GRADIENT 2

typedef struct {
    int32_t iterations;        /* iterations run */
    double final_error;        /* E of the last iteration */
    double *error_history;     /* optional HOST array of max_iter entries (E per iteration) */
    double adjoint_ms;         /* with timing: summed device time of the projection kernels */
    double forward_ms;         /* with timing: summed device time of the dose kernels */
    double update_ms;          /* with timing: summed device time of normalise/update/error */
    double final_ver;          /* V at the last check */
    double *ver_history;       /* optional HOST array of max_iter entries: V at checked iterations, NaN elsewhere */
} vamrt_opt_report;

vamrt_status vamrt_optimize(vamrt_projector *p, const float *target, float *model, void *proj,
                            void *dose, const vamrt_opt_params *params, vamrt_opt_report *report,
                            void *stream);

/*
 * Thresholded dose loss (the differentiable objective around the dose operator; the
 * paper's optimiser targets the same in-part / out-of-part contrast, Sec. 2.7):
 *   L = (1/|P|) sum_P relu(d_h - D)^2 + (1/|Q|) sum_Q relu(D - d_l)^2,
 *   P = {target > 1/2}, Q = the other voxels (|.| counted at least 1),
 * and, if grad is not NULL, dL/dD = -2 relu(d_h - D)/|P| on P, +2 relu(D - d_l)/|Q| on Q.
 * dose: device [nz][ny][nx] in dose_dtype; target: device f32, same layout; loss: DEVICE
 * pointer to one double (FP64 sums in a fixed order: deterministic); grad: device, dose
 * layout, grad_dtype.  Uses the handle's reduction buffer.  Errors: EINVAL, ECUDA.
 */
vamrt_status vamrt_threshold_loss(vamrt_projector *p, const void *dose, vamrt_dtype dose_dtype, const float *target,
                                  double d_l, double d_h, double *loss, void *grad, vamrt_dtype grad_dtype,
                                  void *stream);

/*
 * Voxel error rate (VER) of a dose against a binary target: the fraction of resin voxels
 * (centres within r_inner_mm of the axis) whose printed state differs from the target at
 * the best of the 1023 thresholds tau_i = (i/1024) max(dose), i = 1..1023, max over the
 * resin voxels -- how well the
 * dose prints the part whatever its scale (the optimiser's goal, Sec. 2.7).  A voxel is
 * above tau_i iff min(floor(dose * (1024 / max)), 1023) >= i, evaluated in FP32.
 * dose: device [nz][ny][nx] in dose_dtype (>= 0); target: device f32.  Writes the rate
 * to *ver and the best i to *threshold_index (may be NULL).  Synchronous.
 */
vamrt_status vamrt_voxel_error_rate(vamrt_projector *p, const void *dose, vamrt_dtype dose_dtype, const float *target,
                                    double *ver, int32_t *threshold_index, void *stream);

/*
 * 3x3x3 (taps = 27) or 1x1x1 (taps = 1) convolution, stride 1, zero padding, on the
 * tensor cores: the layers of the learned warm start (a 3D U-Net mapping a target's
 * projections to initial optimiser projections; the paper's optimiser starts from the
 * target itself, Sec. 2.7).  BF16 operands, FP32 accumulation:
 *   y[p][co] = act(bias[co] + sum_{t,ci} x[p + off(t)][ci] w[co][t][ci]),  act = ReLU if relu.
 * x: device [d][h][wd][cin] bf16 (channels last), cin a multiple of 16; w: device
 * [cout][taps][cin] bf16; bias: device f32 [cout] or NULL; y: device [d][h][wd][cout],
 * bf16 (out_f32 = 0) or f32; cout a multiple of 16, <= 256.  x and w 16-byte aligned.
 * err_flag: device int32, set to 1 if a bounded wait inside the kernel timed out (the
 * output is then invalid).  Errors: EINVAL, ECUDA.
 */
vamrt_status vamrt_conv3d_bf16(const void *x, const void *w, const float *bias, void *y, int32_t out_f32, int32_t d,
                               int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps, int32_t relu,
                               int32_t *err_flag, void *stream);

/*
 * Radon-method baseline (Sec. 2.3): projections computed without ray tracing as the
 * parallel-beam Radon transform of every z-slice, a Ram-Lak filter along each sinogram
 * row, and negative values clipped to zero.  The Radon transform is vamrt_adjoint on a
 * projector with parallel chief rays, no refraction and no attenuation (pupil and
 * f-number INFINITY, one ray per pixel, all refractive indices 1, mu = 0); this call is
 * the filter.  Reading of the paper's "Ram-Lak filter in the Fourier domain": the
 * band-limited ramp kernel (unit pitch) h[0] = 1/4, h[n] = -1/(pi^2 n^2) for odd n, 0 for
 * even n != 0, as a linear convolution along the row (zero outside it), equal to the
 * Fourier-domain product on a row padded to twice its length:
 *   out[r][u] = (1 / pixel_mm) sum_{u'} h[u - u'] proj[r][u'],
 * then max(out, 0) when flags has VAMRT_CLAMP_NONNEG.  The paper's coordinate remap for
 * refraction is not applied (its reference is not available).
 * proj, out: device f32 [rows][nu] (out may be proj: filtered in place); nu in 1..4096;
 * rows >= 0 (0: nothing to do); pixel_mm > 0: the detector pitch.  Stream-ordered, no
 * allocation.  Errors: EINVAL (NULL, sizes, pitch, flags, alignment), ECUDA.
 */
vamrt_status vamrt_ramlak_filter(const float *proj, float *out, int64_t rows, int32_t nu, double pixel_mm,
                                 uint32_t flags, void *stream);

/*
 * vamrt_conv3d_tiling: which kernel vamrt_conv3d_bf16 runs for this shape on the current
 * device, written to out[4] (host array): out[0] = 1 for the halo-tile kernel (W % 8 == 0
 * and W <= 240, x 16-byte aligned at run time; regions of out[1] planes x out[2] rows,
 * out[3] output channels per work item), 0 for the
 * gather kernel (out[1..3] = 0).  Host-only query, launches nothing.  Errors: EINVAL (NULL or
 * sizes vamrt_conv3d_bf16 rejects), ECUDA (no device).
 */
vamrt_status vamrt_conv3d_tiling(int32_t d, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                                 int32_t *out);

/*
 * Host-only planning queries (no device, no launch): the tiling the convolution kernels use
 * for a shape on a GPU with `sms` SMs, written to a host array.
 * vamrt_conv3d_halo_plan: out[18] = {planned (0: the gather kernel takes the shape), TZ,
 *   TY, Nt (output channels per work item), T (M tiles per region), WP (slots per staged
 *   row), PT (slots per staged plane), NX (dx taps stacked in N), rowtile, mg (margin
 *   rows), adv (slots between tiles), a_bytes (staged input tile with slack), box_bytes
 *   (its TMA box), stage_bytes, ncols (TMEM), ry (regions along y), nslice, nitems}.
 * vamrt_conv3d_wgrad_plan: out[17] = {planned, Mtot (taps x cin), nmt (M tiles), tpg
 *   (tiles per group), kp (accumulators per tile), KS (positions per stage), BX (positions
 *   per X box), nstage, cwA, cwB (channels per column block of X and dy), slots,
 *   slot_bytes, per_sm (blocks per SM), ncols (TMEM), ngroups, nsplit, spb (stages per
 *   block)}.
 * Errors: EINVAL (NULL out, sms < 1, empty volume); an unsupported shape returns VAMRT_OK
 * with out[0] = 0.
 */
vamrt_status vamrt_conv3d_halo_plan(int32_t d, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                                    int32_t sms, int32_t *out);
vamrt_status vamrt_conv3d_wgrad_plan(int32_t d, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                                     int32_t sms, int32_t *out);


/*
 * Building blocks of the learned warm start (a 3D U-Net on the projection stack; the paper
 * has no such network -- its optimiser starts from the target, Sec. 2.7).  Activations are
 * channels-last BF16 [d][h][w][c] device arrays; gradients of weights and biases are FP32.
 *
 * vamrt_conv3d_wgrad_bf16: dw[co][t][ci] += sum_p dy[p][co] x[p + off(t)][ci] for the
 *   convolution of vamrt_conv3d_bf16 (same x layout; dy [d][h][wd][cout]); tensor cores
 *   (rows t cin + ci in M, cout in N, positions in K; operands loaded by TMA), split over
 *   positions with FP32 atomics (caller zeroes dw).  wd a multiple of 16, d h wd < 2^31,
 *   cin 16..1024, cout 16..256; x and dy 16-byte aligned.
 * vamrt_nn_resample: op 0 = 2x2x2 average pool (fine -> coarse), 1 = its backward (coarse
 *   -> fine, /8), 2 = nearest 2x upsample (coarse -> fine), 3 = its backward (sum of 8);
 *   d, h, w are the FINE extents (even).
 * vamrt_nn_concat: ab[p] = (a[p], b[p]) over channels; backward = 1 splits ab into a, b.
 * vamrt_nn_relu_backward: dy <- dy where y > 0, else 0 (n elements).
 * vamrt_nn_bias_grad: db[c] += sum_p dy[p][c] (c <= 256).
 * vamrt_nn_flip_weights: wt[ci][taps-1-t][co] = w[co][t][ci] (the data-gradient
 *   convolution's weights: dx = conv(dy, wt)).
 * vamrt_nn_adam: Adam step on FP32 params (moments m, v), refreshing an optional BF16 copy.
 * vamrt_nn_prepare_input: x[z][v][u][0] = scale proj[z mod n_angles][v][u] (angles padded
 *   circularly to d_padded), channels 1..15 zero.
 * vamrt_nn_head_mse: residual head on the first n_angles slices, v = in_scale base + z[...][0]
 *   (base: the network's input projections [n_angles][nv][nu] f32); out = out_scale max(v, 0)
 *   (may be NULL); loss = mean 0.5 (v - target_scale target)^2 (device double, may be NULL);
 *   dz (BF16, layout of z, may be NULL) = dloss/dz.
 * vamrt_nn_add: y += x (BF16, n elements).
 * vamrt_projected_step: g <- max(0, g - eta grad) (FP32, n elements).
 * vamrt_projected_adam: one Adam step on projections, kept non-negative:
 *   m <- b1 m + (1-b1) grad; v <- b2 v + (1-b2) grad^2;
 *   g <- max(0, g - lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps)),
 *   and g_bf16 (may be NULL) <- g rounded to BF16 (the storage the operators then read).
 *   FP32 g, grad, m, v of n elements; step >= 1.  The adjoint-driven continuation of the
 *   warm start: grad = A^T dL/dD of the thresholded dose loss.
 * vamrt_nn_absmax: *out = max |x| over n FP32 elements (out: device float).
 * Errors: EINVAL (NULL or bad sizes), ECUDA.
 */
vamrt_status vamrt_conv3d_wgrad_bf16(const void *x, const void *dy, float *dw, int32_t d, int32_t h, int32_t wd,
                                     int32_t cin, int32_t cout, int32_t taps, int32_t *err_flag, void *stream);
vamrt_status vamrt_nn_resample(int32_t op, const void *in, void *out, int32_t d, int32_t h, int32_t w, int32_t c,
                               void *stream);
vamrt_status vamrt_nn_concat(void *a, int32_t ca, void *b, int32_t cb, void *ab, int64_t npos, int32_t backward,
                             void *stream);
vamrt_status vamrt_nn_relu_backward(const void *y, void *dy, int64_t n, void *stream);
vamrt_status vamrt_nn_bias_grad(const void *dy, float *db, int64_t npos, int32_t c, void *stream);
vamrt_status vamrt_nn_flip_weights(const void *w, void *wt, int32_t cout, int32_t taps, int32_t cin, void *stream);
vamrt_status vamrt_nn_adam(float *param, const float *grad, float *m, float *v, void *param_bf16, int64_t n, float lr,
                           float beta1, float beta2, float eps, int32_t step, void *stream);
vamrt_status vamrt_nn_prepare_input(const float *proj, void *x, int32_t n_angles, int32_t nv, int32_t nu,
                                    int32_t d_padded, float scale, void *stream);
vamrt_status vamrt_nn_head_mse(const float *z, int32_t cz, const float *base, float in_scale, const float *target,
                               float target_scale, float *out, float out_scale, void *dz, int32_t n_angles,
                               int32_t nv, int32_t nu, int32_t d_padded, double *loss, void *stream);
vamrt_status vamrt_nn_add(const void *x, void *y, int64_t n, void *stream);
vamrt_status vamrt_projected_step(float *g, const float *grad, float eta, int64_t n, void *stream);
vamrt_status vamrt_projected_adam(float *g, const float *grad, float *m, float *v, void *g_bf16, int64_t n, float lr,
                                  float beta1, float beta2, float eps, int32_t step, void *stream);
vamrt_status vamrt_nn_absmax(const float *x, int64_t n, float *out, void *stream);

/*
 * 8-bit export of projections before the final dose simulation (Sec. 2.7: values more
 * than three standard deviations above the mean are clipped and the range is rescaled
 * to the projector's 8-bit grey levels).  c = mean + 3 sigma over all n_angles x nv x nu
 * values (population sigma, FP64); codes[i] = round-half-even(255 min(max(g,0), c) / c).
 * proj: device, projector layout, proj_dtype; codes: device uint8, same count; dequant:
 * device f32 or NULL, = codes * c / 255 (what the printer delivers, for the final dose);
 * clip: HOST double or NULL (then the call is asynchronous), receives c.
 */
vamrt_status vamrt_export_u8(vamrt_projector *p, const void *proj, vamrt_dtype proj_dtype, uint8_t *codes,
                             float *dequant, double *clip, void *stream);

/*
 * Copy the theta = 0 ray table (kept in FP64 on the device), rounded to FP32, to HOST
 * arrays of n_rays entries each (ray index r = (a nv + v) nu + u):  a4[r] = (e_x, e_y, e_z, delta) in voxel units (entry point
 * relative to the axis, sample spacing);  b4[r] = (d_x, d_y, d_z, T1 T2 delta_mm / M);
 * j2[r] = (j_lo, j_hi), the samples whose footprint reaches the grid (-1 < q_z < nz).
 * Any pointer may be NULL.  Synchronous.
 */
vamrt_status vamrt_copy_ray_table(const vamrt_projector *p, float *a4, float *b4, int32_t *j2);

/*
 * Measured shared-memory read bandwidth of the current device in bytes/s (conflict-free
 * 32-bit volatile loads on every SM, none merged or dropped).  The operators stage their per-sample corner words in shared
 * memory, so this is the denominator of their roofline.  Synchronises `stream`; allocates
 * a small temporary device buffer.  Errors: EINVAL (NULL), ENOMEM, ECUDA.
 */
vamrt_status vamrt_measure_smem_bandwidth(double *bytes_per_second, void *stream);

/*
 * Measured L2 rates of the current device: *read_bytes_per_second for 16-byte loads that
 * bypass L1 over a 32 MiB buffer resident in L2, and *red_ops_per_second for 16-byte
 * vector reductions (red.global.add.v4.f32, the dose flush's instruction) to distinct
 * addresses of that buffer.  The operators stage volume boxes from L2 and flush dose
 * boxes into it, so these bound their L2 traffic.  Synchronises `stream`; allocates a
 * temporary 32 MiB device buffer.  Errors: EINVAL (NULL), ENOMEM, ECUDA.
 */
vamrt_status vamrt_measure_l2_rates(double *read_bytes_per_second, double *red_ops_per_second, void *stream);

/* Number of kernels this library has launched in the process (all devices). */
uint64_t vamrt_launch_count(void);

/* Static description of a status code. */
const char *vamrt_status_string(vamrt_status s);

/* Detail of the last error on the calling thread ("" if none). */
const char *vamrt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VAMRT_H */
