// Dose operator whose FP32 accumulator lives in a statically allocated device array.
//
// vamrt_forward_dose sums into a scratch volume that vamrt_make_projector allocated with
// cudaMalloc.  Some callers cannot allocate device memory at all -- a host process whose
// device memory is owned by another allocator or budgeted up front, or code that must
// not trigger an allocation (and the device synchronisation it can imply) at the point
// of the call.  This variant runs the same kernels with the accumulator in a file-scope
// __device__ array of fixed size, so the call itself allocates nothing: no cudaMalloc,
// no cudaFree, no library routine that allocates.
#include <stdio.h>

#include <cuda.h>

#include <mutex>

#include "internal.cuh"

namespace {

// 4 Mi floats = 16 MiB: padded grids of up to (nx+2, rounded up to a multiple of 4) x
// (ny+2) x (nz+2) = 4,194,304 voxels (e.g. up to 158^3).  Every device that loads the
// library holds this array until the process exits.
constexpr int64_t kStaticAccFloats = 4 * 1024 * 1024;
static __device__ __align__(256) float g_static_acc[kStaticAccFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the context the address was looked up in, and the address.
void *g_acc_ctx[kMaxDevices] = {};
float *g_acc_addr[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

// The driver's cuCtxGetCurrent, through the runtime's entry-point query (the library links
// the static runtime only).  NULL when the driver does not provide it.
CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
    });
    return fn;
}

}  // namespace

namespace vamrt {

// Device address of g_static_acc on the current device (dev).  In host code the array's
// name is only a host-side stand-in, so the address must come from the runtime, with the
// device current.  Looking it up also loads the array's module (the library's modules load
// lazily), which is what allocates the array on the device; vamrt_make_projector calls
// this so that the allocation happens there and not in vamrt_forward_dose_static.  The
// address is cached per device together with the context it was found in, and looked up
// again when the current context differs (after a device reset).
cudaError_t static_acc_address(int dev, float **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    CUcontext ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get) get(&ctx);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_acc_addr[dev] || g_acc_ctx[dev] != (void *)ctx) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_acc);
        if (e != cudaSuccess) return e;
        g_acc_addr[dev] = (float *)ptr;
        g_acc_ctx[dev] = (void *)ctx;
    }
    *out = g_acc_addr[dev];
    return cudaSuccess;
}

}  // namespace vamrt

extern "C" vamrt_status vamrt_forward_dose_static(const vamrt_projector *p, const void *proj,
                                                  vamrt_dtype proj_dtype, void *dose, vamrt_dtype dose_dtype,
                                                  uint32_t flags, void *stream)
{
    char msg[256];
    if (!p || !proj || !dose) {
        snprintf(msg, sizeof(msg), "NULL argument");
        vamrt::set_error(msg);
        return VAMRT_EINVAL;
    }
    if ((proj_dtype != VAMRT_F32 && proj_dtype != VAMRT_BF16) || (dose_dtype != VAMRT_F32 && dose_dtype != VAMRT_BF16)) {
        snprintf(msg, sizeof(msg), "unknown dtype");
        vamrt::set_error(msg);
        return VAMRT_EINVAL;
    }
    if (flags & ~VAMRT_ACCUMULATE) {
        snprintf(msg, sizeof(msg), "unknown flags 0x%x", flags);
        vamrt::set_error(msg);
        return VAMRT_EINVAL;
    }
    if (p->pad_elems > kStaticAccFloats) {
        snprintf(msg, sizeof(msg),
                 "grid too large for the static accumulator: %lld padded voxels, maximum %lld",
                 (long long)p->pad_elems, (long long)kStaticAccFloats);
        vamrt::set_error(msg);
        return VAMRT_EINVAL;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        snprintf(msg, sizeof(msg), "no usable current device");
        vamrt::set_error(msg);
        return VAMRT_ECUDA;
    }
    if (dev != p->device) {
        snprintf(msg, sizeof(msg), "current device %d is not the projector's device %d", dev,
                 p->device);
        vamrt::set_error(msg);
        return VAMRT_EINVAL;
    }
    float *acc = nullptr;
    cudaError_t e = vamrt::static_acc_address(dev, &acc);
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear the part this grid uses
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(float) * p->pad_elems, s);
    if (e == cudaSuccess) e = vamrt::launch_forward_acc(p, proj, proj_dtype, acc, s);
    if (e == cudaSuccess) e = vamrt::launch_unpad_acc(p, acc, dose, dose_dtype, flags, s);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "%s", cudaGetErrorString(e));
        vamrt::set_error(msg);
        return VAMRT_ECUDA;
    }
    return VAMRT_OK;
}
