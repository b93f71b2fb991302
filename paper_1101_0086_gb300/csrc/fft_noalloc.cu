// mpa_fft_noalloc: the transform of mpa_fft for callers that cannot hand the
// library a device workspace.
//
// Some callers cannot call cudaMalloc at the point where they need a
// transform: a plugin running inside a host application that owns every
// byte of device memory through its own pool, or a latency-critical loop
// that must not stall on an allocation.  For them this entry point takes
// only the data buffer.  Its scratch is the file-scope array below, which
// every GPU that loads this library holds (MPA_FFT_NOALLOC_MAX_BYTES) until
// the process exits.  The entry point itself allocates nothing.
#include <mutex>

#include "host.h"

using namespace mpa;
using namespace mpa::host;

// Scratch of the no-allocation transform: one N-sample buffer that receives
// the transposed field.  Every call (any stream, any thread) uses the same
// array and leaves the last call's samples in it; calls that overlap on
// the GPU therefore race and must be ordered by the caller.  Nothing in it
// needs to start at zero: each call overwrites the N samples it reads.
static __device__ __align__(256) unsigned char mpa_fft_noalloc_scratch[MPA_FFT_NOALLOC_MAX_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the scratch on the current device.  The array's name is
// only a host-side stand-in, so the address is looked up with the device
// current.  Outside stream capture it is looked up on every call (cheap, and
// it allocates nothing), so a context that was reset and recreated is
// picked up; while `st` is being captured the address cached by the last
// uncaptured call on this device is used (the lookup is not a stream
// operation, but a first call under capture has nothing to fall back on).
cudaError_t scratch_on_current_device(cudaStream_t st, void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, mpa_fft_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = p;
    } else if (!g_scratch[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int mpa_fft_noalloc(int64_t N, int32_t precision, int32_t sign, void* data, mpa_stream stream) {
    if (!data || (sign != 1 && sign != -1)) return MPA_ERR_INVALID_ARG;
    if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
    // the same split as mpa_fft (split_n), checked before the size limit
    Split s;
    int rc = split_n(N, precision, &s);
    if (rc) return rc;
    const size_t bytes = (size_t)N * (precision == MPA_FP32 ? sizeof(float2) : sizeof(double2));
    if (bytes > (size_t)MPA_FFT_NOALLOC_MAX_BYTES) return MPA_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    MPA_TRY(scratch_on_current_device(st, &scratch));
    // the launch sequence of mpa_fft, with the static scratch as its workspace
    if (precision == MPA_FP32) {
        float2* d = reinterpret_cast<float2*>(data);
        float2* w = reinterpret_cast<float2*>(scratch);
        rc = sign > 0 ? fft_forward<float>(s, d, w, st) : fft_inverse<float>(s, d, w, st);
    } else {
        double2* d = reinterpret_cast<double2*>(data);
        double2* w = reinterpret_cast<double2*>(scratch);
        rc = sign > 0 ? fft_forward<double>(s, d, w, st) : fft_inverse<double>(s, d, w, st);
    }
    if (rc) return rc;
    MPA_TRY(cudaMemcpyAsync(data, scratch, bytes, cudaMemcpyDeviceToDevice, st));
    return MPA_OK;
}
