// gempe_fit_sigma_static: the slope fit of gempe_fit_sigma without any device
// allocation.
//
// gempe_fit_sigma stages the caller's histogram in a temporary device buffer
// it allocates per call.  Some callers cannot allocate device memory at that
// point: code running inside another allocator's callbacks (an allocation
// there re-enters the allocator), latency-critical serving loops where
// cudaMalloc / cudaFree would synchronise the device, and processes whose
// device memory is already reserved by a framework's caching allocator (a
// raw cudaMalloc fails there although the framework holds free blocks).  This
// variant stages the histogram in a fixed static device array instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its 32 KiB until the process exits.  In host code the
// array's name is only a host-side stand-in, so its device address is looked
// up with cudaGetSymbolAddress, once per device, with that device current;
// the first call on a device does this look-up (and uploads the Mills-ratio
// table if no context did so before), so that first call should come before
// any stream capture.  All calls share the one array and it keeps the last
// call's contents; nothing in it has to start at zero (each call overwrites
// the histogram part and the kernel writes sigma before it is read back), but
// calls whose work overlaps on the GPU race on the array and must not be
// issued concurrently.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "engine.cuh"
#include "gempe.h"

#define GEMPE_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kStaticMaxBins = 4096;

// [0, 2*bins): edge bins then non-edge bins; [2*kStaticMaxBins]: the result.
static __device__ __align__(256) float g_fit_scratch[2 * kStaticMaxBins + 4];

gempe_status static_fail(gempe_status st, const std::string& msg) {
    gempe::set_last_error(msg.c_str());   // reported by gempe_last_error()
    return st;
}

// Device address of g_fit_scratch on the current device (looked up once per device).
cudaError_t scratch_address(float** out) {
    static std::mutex mu;
    static std::vector<float*> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        float* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_fit_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *out = addr[dev];
    return cudaSuccess;
}

}  // namespace

GEMPE_API gempe_status gempe_fit_sigma_static(const float* host_hist, int32_t bins, float hist_max, float mu,
                                              void* cuda_stream, float* out_sigma) {
    if (!host_hist || !out_sigma) return static_fail(GEMPE_E_INVALID_ARG, "null argument");
    if (bins < 16 || bins > kStaticMaxBins)
        return static_fail(GEMPE_E_INVALID_ARG,
                           "bins must be in [16, 4096]: the static scratch holds at most 4096 bins per side");
    if (!(hist_max > 0.0f) || !std::isfinite(mu))
        return static_fail(GEMPE_E_INVALID_ARG, "hist_max must be positive and mu finite");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = gempe::ensure_mills_table();
    float* d = nullptr;
    if (e == cudaSuccess) e = scratch_address(&d);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d, host_hist, sizeof(float) * 2 * (size_t)bins, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = gempe::launch_fit_sigma(d, bins, hist_max, mu, d + 2 * kStaticMaxBins, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_sigma, d + 2 * kStaticMaxBins, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return static_fail(GEMPE_E_CUDA, std::string("gempe_fit_sigma_static: ") + cudaGetErrorString(e));
    return GEMPE_OK;
}
