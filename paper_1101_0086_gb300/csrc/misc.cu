// Launchers of the scan, transpose and precision-conversion kernels.
#include "launch.h"

namespace mpa {

std::atomic<long long> g_launches{0};

static unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T> cudaError_t scan_launch(const ScanParams<T>& p, cudaStream_t st) {
    scan_kernel<T><<<blocks_for(p.N, 256), 256, 0, st>>>(p);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t transpose_launch(const cx<T>* in, cx<T>* out, long long R, long long C, cudaStream_t st) {
    dim3 grid((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32));
    transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(in, out, R, C);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t to_state_launch(const cx<T>* in, double2* state, cx<T>* copy, long long N, cudaStream_t st) {
    to_state_kernel<T><<<blocks_for(N, 256), 256, 0, st>>>(in, state, copy, N);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T> cudaError_t from_state_launch(const double2* state, cx<T>* out, long long N, cudaStream_t st) {
    from_state_kernel<T><<<blocks_for(N, 256), 256, 0, st>>>(state, out, N);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template cudaError_t scan_launch<float>(const ScanParams<float>&, cudaStream_t);
template cudaError_t scan_launch<double>(const ScanParams<double>&, cudaStream_t);
template cudaError_t transpose_launch<float>(const float2*, float2*, long long, long long, cudaStream_t);
template cudaError_t transpose_launch<double>(const double2*, double2*, long long, long long, cudaStream_t);
template cudaError_t to_state_launch<float>(const float2*, double2*, float2*, long long, cudaStream_t);
template cudaError_t to_state_launch<double>(const double2*, double2*, double2*, long long, cudaStream_t);
template cudaError_t from_state_launch<float>(const double2*, float2*, long long, cudaStream_t);
template cudaError_t from_state_launch<double>(const double2*, double2*, long long, cudaStream_t);

}  // namespace mpa
