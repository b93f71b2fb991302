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

#include "launch.h"
#include "mpa.h"

using namespace mpa;

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
// only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached.
cudaError_t scratch_on_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, mpa_fft_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

int log2_exact(long long n) {
    int l = 0;
    while ((1ll << l) < n) ++l;
    return (1ll << l) == n ? l : -1;
}

template <typename T>
cudaError_t transform(long long N, int logN, int logN1, int logN2, int sign, cx<T>* data, cx<T>* scratch,
                      cudaStream_t st) {
    const long long N1 = 1ll << logN1, N2 = 1ll << logN2;
    cudaError_t e;
    KCParams<T> c{};
    c.dst = sign > 0 ? scratch : data;
    c.src = c.dst;
    c.N = N;
    c.logN = logN;
    c.N1 = (int)N1;
    c.logN1 = logN1;
    c.ncols = N1;
    KRParams<T> r{sign > 0 ? scratch : data, N2, N, logN, (int)N2, (T)(1.0 / (double)N), T(0)};
    if (sign > 0) {
        // natural A(t) (N1 x N2) -> rows of the work layout -> natural spectrum
        if ((e = transpose_launch<T>(data, scratch, N1, N2, st)) != cudaSuccess) return e;
        if ((e = kr_launch<T>(KR_FWD, logN1, r, st)) != cudaSuccess) return e;
        if ((e = kc_launch<T>(KC_FWD, logN2, c, st)) != cudaSuccess) return e;
    } else {
        if ((e = kc_launch<T>(KC_INV, logN2, c, st)) != cudaSuccess) return e;
        if ((e = kr_launch<T>(KR_INV, logN1, r, st)) != cudaSuccess) return e;
        if ((e = transpose_launch<T>(data, scratch, N2, N1, st)) != cudaSuccess) return e;
    }
    return cudaMemcpyAsync(data, scratch, (size_t)N * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st);
}

}  // namespace

extern "C" int mpa_fft_noalloc(int64_t N, int32_t precision, int32_t sign, void* data, mpa_stream stream) {
    if (!data || (sign != 1 && sign != -1)) return MPA_ERR_INVALID_ARG;
    if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
    const int logN = log2_exact((long long)N);
    if (logN < 8 || logN > (precision == MPA_FP32 ? 25 : 24)) return MPA_ERR_UNSUPPORTED_N;
    const size_t csize = precision == MPA_FP32 ? sizeof(float2) : sizeof(double2);
    if ((size_t)N * csize > (size_t)MPA_FFT_NOALLOC_MAX_BYTES) return MPA_ERR_WORKSPACE;
    const int logN2 = logN / 2 < KC_LOG_MAX ? logN / 2 : KC_LOG_MAX;
    const int logN1 = logN - logN2;
    void* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return MPA_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e =
        precision == MPA_FP32
            ? transform<float>(N, logN, logN1, logN2, sign, reinterpret_cast<float2*>(data),
                               reinterpret_cast<float2*>(scratch), st)
            : transform<double>(N, logN, logN1, logN2, sign, reinterpret_cast<double2*>(data),
                                reinterpret_cast<double2*>(scratch), st);
    return e == cudaSuccess ? MPA_OK : MPA_ERR_CUDA;
}
