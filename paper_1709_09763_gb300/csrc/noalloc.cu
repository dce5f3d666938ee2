// Systematic resampling that allocates nothing (C ABI, see include/mls2mc.h).
//
// Some callers cannot allocate device memory: code running inside a framework that owns all
// device memory through its own pool, a host that forbids cudaMalloc after start-up (a
// real-time or embedded loop, where an allocation may block or fail at the worst moment), or a
// plug-in without a handle of this library. For them this entry point keeps its scratch -- the
// cumulative normalised weights, one double per particle -- in a fixed file-scope device array
// instead of memory from cudaMalloc. Every GPU that loads the library holds that array
// (kNoallocMaxParticles doubles) until the process exits.
//
// Host code must not use the array's name as a device address (in host code it only names a
// host-side stand-in): every call looks the address up with cudaGetSymbolAddress, with the
// caller's device current. The address belongs to the CUDA context that loaded the library's
// device code, not to a device ordinal, so it is never cached: after a cudaDeviceReset, or under
// another context made current by the caller, the lookup returns that context's address. The
// first call on a device (and the first after a reset) may load the device code; make it before
// any stream capture: a first call on a capturing stream is refused with SMC_EINVAL. All calls
// share the array and it keeps the last call's contents; the kernels write every entry they read
// before reading it, so nothing needs clearing, but calls that overlap on the GPU (different
// streams, or concurrent host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "smc_device.h"

namespace mls2mc {

namespace {

constexpr int kNoallocMaxParticles = SMC_NOALLOC_MAX_PARTICLES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_cdf_scratch[kNoallocMaxParticles];

std::mutex g_setup_mu;
bool g_loaded[kMaxDevices] = {};   // a lookup has succeeded on this ordinal (device code loaded)

// device address of the scratch array in the current context, looked up on every call
cudaError_t scratch_on_current_device(cudaStream_t stream, double** out, bool* capturing_first) {
    *capturing_first = false;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_loaded[dev]) {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(stream, &st);
        if (e != cudaSuccess) return e;
        if (st != cudaStreamCaptureStatusNone) {
            *capturing_first = true;
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cdf_scratch);
    if (e != cudaSuccess) return e;
    g_loaded[dev] = true;
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace

}  // namespace mls2mc

extern "C" int smc_systematic_resample_noalloc(const double* w, int n, double U, int* anc, void* stream) {
    using namespace mls2mc;
    if (n < 1 || n > kNoallocMaxParticles) return SMC_EINVAL;   // beyond the fixed scratch: rejected
    if (!w || !anc || !(U >= 0.0 && U < 1.0)) return SMC_EINVAL;
    double* cdf = nullptr;
    bool capturing_first = false;
    cudaError_t e = scratch_on_current_device(static_cast<cudaStream_t>(stream), &cdf, &capturing_first);
    if (e != cudaSuccess) return SMC_ECUDA;
    if (capturing_first) return SMC_EINVAL;   // first call on this device made during a stream capture
    e = resample_launch(nullptr, w, n, nullptr, U, 0u, 0ull, cdf, anc, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}
