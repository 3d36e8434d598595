// plk_static.cu -- an evaluation entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they evaluate:
// plugins whose host application owns the whole device-memory budget, and
// latency-critical loops that must not call cudaMalloc/cudaFree because those
// calls can stall or synchronize work running elsewhere on the device.  For
// them, this file keeps the scratch memory the pipeline needs in one
// file-scope device array, reserved when the library's module is loaded and
// held by every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "plk.h"
#include "plk_kernels.cuh"

namespace {

// The scratch array itself.  In host code `g_scratch` names a host-side
// stand-in, not device memory: its device address comes from
// cudaGetSymbolAddress, looked up once per device below.
static __device__ __align__(256) unsigned char g_scratch[PLK_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

}  // namespace

extern "C" plk_status plk_eval_device_static(const plk_eval_args *args, int32_t reml, void *stream) {
    if (!args) {
        plk::set_last_error("plk_eval_device_static: args is NULL");
        return PLK_E_INVALID;
    }
    // Largest batch whose workspace fits in the array; reject sizes for which
    // even one point does not fit.
    const size_t one = plk_eval_workspace_bytes(args->n, args->p, args->M, 1, PLK_FP64);
    if (one == 0) return plk_eval_device(args, nullptr, nullptr, 0, stream);   // reports the size error
    if (one > (size_t)PLK_STATIC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "plk_eval_device_static: n=%lld needs %zu bytes of scratch for one point; the static "
                 "scratch holds %zu bytes (use plk_eval_device with a caller workspace)",
                 (long long)args->n, one, (size_t)PLK_STATIC_SCRATCH_BYTES);
        plk::set_last_error(buf);
        return PLK_E_NOMEM;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        plk::set_last_error((std::string("plk_eval_device_static: cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
        return PLK_E_CUDA;
    }
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            // set-up, once per device, with that device current
            e = cudaGetSymbolAddress(&g_addr[dev], g_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                plk::set_last_error(
                    (std::string("plk_eval_device_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
                return PLK_E_CUDA;
            }
        }
        ptr = g_addr[dev];
    }
    int32_t batch = 1;
    while (batch < args->K &&
           plk_eval_workspace_bytes(args->n, args->p, args->M, batch * 2, PLK_FP64) <= (size_t)PLK_STATIC_SCRATCH_BYTES)
        batch *= 2;
    while (batch > 1 && plk_eval_workspace_bytes(args->n, args->p, args->M, batch, PLK_FP64) > (size_t)PLK_STATIC_SCRATCH_BYTES)
        batch -= 1;
    plk_options o{};
    o.precision = PLK_FP64;
    o.reml = reml;
    o.batch = batch;
    o.flags = 0;
    return plk_eval_device(args, &o, ptr, (size_t)PLK_STATIC_SCRATCH_BYTES, stream);
}
