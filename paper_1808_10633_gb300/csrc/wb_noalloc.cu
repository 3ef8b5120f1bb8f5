// wb_noalloc.cu -- conserved totals over a caller-owned device state without
// any allocation (wb_conserved_totals_noalloc).
//
// Some callers cannot allocate device memory: code that runs under another
// component's memory pool (a framework that owns every byte of the device
// and forbids out-of-band cudaMalloc), or a time-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// For them this entry point runs the same two-pass deterministic reduction
// as wb_conserved_totals, with its per-block partial sums in a file-scope
// device array instead of memory allocated by the library.
//
// The scratch array below is created when the library is loaded and held by
// every GPU that loads the library until the process exits (64 KiB each).
// Host code must not pass the symbol itself to a kernel: on the host the
// name is a stand-in, not a device address.  The device address is looked up
// with cudaGetSymbolAddress, with the caller's device current, on every call
// outside stream capture.
#include "../../include/wombat_gb300.h"
#include "wb_internal.h"

#include <mutex>

namespace {

constexpr int kNoAllocPartials = WB_NOALLOC_PARTIALS;

// Per-block partial sums (8 doubles per block) of the two-pass reduction.
static __device__ __align__(256) double g_noalloc_partial[kNoAllocPartials * 8];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Looked up
// again on every call whose stream is not being captured, so that a
// cudaDeviceReset between calls (which unloads the module and may place the
// array elsewhere when it is loaded again) leaves no stale address; while
// the stream is being captured, the address of the last call outside
// capture on this device is used.
cudaError_t scratch_address(cudaStream_t s, double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<double*>(p);
    } else if (!g_scratch[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int wb_conserved_totals_noalloc(const void* state, int precision, long long ncells,
                                           double dV, double* out, void* cuda_stream) {
    if (!state || !out) return wb::set_last_error(WB_EINVAL, "noalloc totals: null state or out");
    if (precision != WB_FP64 && precision != WB_FP32)
        return wb::set_last_error(WB_EINVAL, "noalloc totals: unknown precision");
    if (ncells < 1 || ncells > WB_NOALLOC_MAX_CELLS)
        return wb::set_last_error(WB_EINVAL,
                                  "noalloc totals: ncells must be in [1, WB_NOALLOC_MAX_CELLS = 2^34]");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* partial = nullptr;
    cudaError_t se = scratch_address(s, &partial);
    if (se == cudaErrorStreamCaptureUnsupported)
        return wb::set_last_error(WB_EINVAL, "noalloc totals: the first call on a device must come "
                                             "before any stream capture");
    if (se != cudaSuccess)
        return wb::set_last_error(WB_ECUDA, "noalloc totals: scratch address lookup failed");
    // Every one of the kNoAllocPartials partial slots is rewritten by pass 1
    // (blocks with an empty chunk write zeros), so nothing is cleared first.
    cudaError_t e;
    if (precision == WB_FP64)
        e = wb::launch_totals<double>(static_cast<const double*>(state), nullptr, 0, ncells,
                                      partial, kNoAllocPartials, dV, out, s);
    else
        e = wb::launch_totals<float>(static_cast<const float*>(state), nullptr, 0, ncells,
                                     partial, kNoAllocPartials, dV, out, s);
    if (e != cudaSuccess) return wb::set_last_error(WB_ECUDA, "noalloc totals: kernel launch failed");
    return wb::set_last_error(WB_OK, "");
}
