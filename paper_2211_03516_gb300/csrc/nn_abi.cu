// C-ABI entry points of the warm-start network's building blocks (tensor-core weight
// gradient, resampling, concatenation, ReLU/bias gradients, weight flip, Adam, input and
// head kernels) and of the projected-gradient step.  Argument checks only; all work runs
// in the kernels of conv3d_tc.cu and nn_ops.cu.
#include <stdint.h>

#include "internal.cuh"

namespace {
vamrt_status einval(const char *msg)
{
    vamrt::set_error(msg);
    return VAMRT_EINVAL;
}
vamrt_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return VAMRT_OK;
    vamrt::set_error(cudaGetErrorString(e));
    return VAMRT_ECUDA;
}
}  // namespace

extern "C" {

vamrt_status vamrt_conv3d_wgrad_bf16(const void *x, const void *dy, float *dw, int32_t d, int32_t h, int32_t wd,
                                     int32_t cin, int32_t cout, int32_t taps, int32_t *err_flag, void *stream)
{
    if (!x || !dy || !dw || !err_flag) return einval("NULL argument");
    if (d < 1 || h < 1 || wd < 16 || wd % 16) return einval("extents: d, h >= 1 and wd a multiple of 16");
    if ((int64_t)d * h * wd >= ((int64_t)1 << 31)) return einval("d h wd must stay below 2^31 positions");
    if (cin < 16 || cin % 16 || cin > 1024 || cout < 16 || cout % 16 || cout > 256)
        return einval("channel counts: cin 16..1024, cout 16..256, multiples of 16");
    if (taps != 1 && taps != 27) return einval("taps must be 1 or 27");
    if (((uintptr_t)x | (uintptr_t)dy) & 15) return einval("x and dy must be 16-byte aligned");
    return cuda_status(vamrt::launch_conv3d_wgrad_tc(x, dy, dw, d, h, wd, cin, cout, taps, (int *)err_flag,
                                                     (cudaStream_t)stream));
}

vamrt_status vamrt_conv3d_halo_plan(int32_t d, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                                    int32_t sms, int32_t *out)
{
    if (!out || sms < 1 || d < 1 || h < 1 || wd < 1) return einval("NULL out, sms < 1 or empty volume");
    vamrt::ConvHaloPlan pl;
    for (int i = 0; i < 18; ++i) out[i] = 0;
    if (!vamrt::plan_conv3d_halo(d, h, wd, cin, cout, taps, sms, &pl)) return VAMRT_OK;
    const int32_t v[18] = {1, pl.TZ, pl.TY, pl.Nt, pl.T, pl.WP, pl.PT, pl.NX, pl.rowtile, pl.mg, pl.adv,
                           pl.a_bytes, pl.box_bytes, pl.stage_bytes, pl.ncols, pl.ry, pl.nslice, pl.nitems};
    for (int i = 0; i < 18; ++i) out[i] = v[i];
    return VAMRT_OK;
}

vamrt_status vamrt_conv3d_wgrad_plan(int32_t d, int32_t h, int32_t wd, int32_t cin, int32_t cout, int32_t taps,
                                     int32_t sms, int32_t *out)
{
    if (!out || sms < 1 || d < 1 || h < 1 || wd < 1) return einval("NULL out, sms < 1 or empty volume");
    vamrt::WgradPlan pl;
    for (int i = 0; i < 17; ++i) out[i] = 0;
    if (!vamrt::plan_wgrad_tma(d, h, wd, cin, cout, taps, sms, &pl)) return VAMRT_OK;
    const int32_t v[17] = {1, pl.Mtot, pl.nmt, pl.tpg, pl.kp, pl.KS, pl.BX, pl.nstage, pl.cwA, pl.cwB,
                           pl.slots, pl.slot_bytes, pl.per_sm, pl.ncols, pl.ngroups, pl.nsplit, pl.spb};
    for (int i = 0; i < 17; ++i) out[i] = v[i];
    return VAMRT_OK;
}

vamrt_status vamrt_nn_resample(int32_t op, const void *in, void *out, int32_t d, int32_t h, int32_t w, int32_t c,
                               void *stream)
{
    if (!in || !out) return einval("NULL argument");
    if (op < 0 || op > 3) return einval("op must be 0..3");
    if (d < 2 || h < 2 || w < 2 || (d | h | w) & 1 || c < 1) return einval("fine extents must be even and >= 2");
    return cuda_status(vamrt::nn_resample(op, in, out, d, h, w, c, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_concat(void *a, int32_t ca, void *b, int32_t cb, void *ab, int64_t npos, int32_t backward,
                             void *stream)
{
    if (!a || !b || !ab) return einval("NULL argument");
    if (ca < 1 || cb < 1 || npos < 0) return einval("sizes");
    return cuda_status(vamrt::nn_concat(a, ca, b, cb, ab, npos, backward, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_relu_backward(const void *y, void *dy, int64_t n, void *stream)
{
    if (!y || !dy || n < 0) return einval("bad argument");
    return cuda_status(vamrt::nn_relu_bwd(y, dy, n, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_bias_grad(const void *dy, float *db, int64_t npos, int32_t c, void *stream)
{
    if (!dy || !db || npos < 0 || c < 1 || c > 256) return einval("bad argument");
    return cuda_status(vamrt::nn_bias_grad(dy, db, npos, c, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_flip_weights(const void *w, void *wt, int32_t cout, int32_t taps, int32_t cin, void *stream)
{
    if (!w || !wt || cout < 1 || cin < 1 || (taps != 1 && taps != 27)) return einval("bad argument");
    return cuda_status(vamrt::nn_flip_weights(w, wt, cout, taps, cin, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_adam(float *param, const float *grad, float *m, float *v, void *param_bf16, int64_t n, float lr,
                           float beta1, float beta2, float eps, int32_t step, void *stream)
{
    if (!param || !grad || !m || !v || n < 0 || step < 1) return einval("bad argument");
    return cuda_status(vamrt::nn_adam(param, grad, m, v, param_bf16, n, lr, beta1, beta2, eps, step, false,
                                      (cudaStream_t)stream));
}

vamrt_status vamrt_projected_adam(float *g, const float *grad, float *m, float *v, void *g_bf16, int64_t n, float lr,
                                  float beta1, float beta2, float eps, int32_t step, void *stream)
{
    if (!g || !grad || !m || !v || n < 0 || step < 1) return einval("bad argument");
    if (!(lr >= 0.f) || !(eps > 0.f)) return einval("lr must be >= 0 and eps > 0");
    return cuda_status(vamrt::nn_adam(g, grad, m, v, g_bf16, n, lr, beta1, beta2, eps, step, true,
                                      (cudaStream_t)stream));
}

vamrt_status vamrt_nn_prepare_input(const float *proj, void *x, int32_t n_angles, int32_t nv, int32_t nu,
                                    int32_t d_padded, float scale, void *stream)
{
    if (!proj || !x || n_angles < 1 || nv < 1 || nu < 1 || d_padded < n_angles) return einval("bad argument");
    return cuda_status(vamrt::nn_prepare_input(proj, x, n_angles, nv, nu, d_padded, scale, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_head_mse(const float *z, int32_t cz, const float *base, float in_scale, const float *target,
                               float target_scale, float *out, float out_scale, void *dz, int32_t n_angles,
                               int32_t nv, int32_t nu, int32_t d_padded, double *loss, void *stream)
{
    if (!z || !base || cz < 1 || n_angles < 1 || nv < 1 || nu < 1 || d_padded < n_angles) return einval("bad argument");
    return cuda_status(vamrt::nn_head_mse(z, cz, base, in_scale, target, target_scale, out, out_scale, dz, n_angles,
                                          nv, nu, d_padded, loss, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_add(const void *x, void *y, int64_t n, void *stream)
{
    if (!x || !y || n < 0) return einval("bad argument");
    return cuda_status(vamrt::nn_add(x, y, n, (cudaStream_t)stream));
}

vamrt_status vamrt_projected_step(float *g, const float *grad, float eta, int64_t n, void *stream)
{
    if (!g || !grad || n < 0) return einval("bad argument");
    return cuda_status(vamrt::nn_projected_step(g, grad, eta, n, (cudaStream_t)stream));
}

vamrt_status vamrt_nn_absmax(const float *x, int64_t n, float *out, void *stream)
{
    if (!x || !out || n < 0) return einval("bad argument");
    return cuda_status(vamrt::nn_absmax(x, n, out, (cudaStream_t)stream));
}

}  // extern "C"
