// mpa_alu_peak: measured FMA throughput of the current GPU in FP64 or FP32,
// the denominator of the ALU-bound roofline of the split-step comparator.
//
// Every thread runs 8 independent chains x = x a + b of fused multiply-adds
// (enough independent work to cover the FMA latency at full occupancy), so
// the kernel's time is set by the FMA issue rate alone.  Nothing is read or
// written in global memory except one value per block, stored only when it
// can never match (keeps the compiler from removing the chains).
#include "host.h"

namespace {

__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(int reps, T a, T b) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (T)(threadIdx.x + u) * (T)1e-3;
#pragma unroll 8
    for (int r = 0; r < reps; ++r) {  // reps is a multiple of 8
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == (T)-1.2345e30) g_peak_sink = (double)s;
}

template <typename T>
int run(double* flops, cudaStream_t st) {
    int dev = 0, sms = 0;
    MPA_TRY(cudaGetDevice(&dev));
    MPA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned blocks = (unsigned)sms * 8u;  // 8 x 256 threads per SM: full occupancy
    const int reps = sizeof(T) == 8 ? 4096 : 65536;
    // a close to 1 and b small keep x finite for any reps
    const T a = (T)0.999999, b = (T)1e-6;
    cudaEvent_t e0, e1;
    MPA_TRY(cudaEventCreate(&e0));
    MPA_TRY(cudaEventCreate(&e1));
    float best = -1.f;
    int rc = MPA_OK;
    for (int it = 0; it < 4 && rc == MPA_OK; ++it) {  // the first run warms up
        if (const cudaError_t eg = mpa::launch_gate()) {
            rc = mpa::host::cuda_fail(eg);
            break;
        }
        cudaError_t e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fma_chains_kernel<T><<<blocks, 256, 0, st>>>(reps, a, b);
            mpa::g_launches.fetch_add(1, std::memory_order_relaxed);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = mpa::host::cuda_fail(e);
        else if (it > 0 && (best < 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MPA_OK) return rc;
    *flops = 2.0 * 8.0 * (double)reps * (double)blocks * 256.0 / (best * 1e-3);
    return MPA_OK;
}

}  // namespace

extern "C" int mpa_alu_peak(int32_t precision, double* flops_per_s, mpa_stream stream) {
    if (!flops_per_s || (precision != MPA_FP32 && precision != MPA_FP64)) return MPA_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return precision == MPA_FP64 ? run<double>(flops_per_s, st) : run<float>(flops_per_s, st);
}
