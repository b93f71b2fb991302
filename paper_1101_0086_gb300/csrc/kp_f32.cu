// Launcher of the persistent batch kernel (FP32, on-chip node transform).
#include "kp.cuh"
#include "launch.h"

namespace mpa {

// Tags of a fresh queue (slot i: i) and zero counters, before kp_kernel.
__global__ void __launch_bounds__(256) kp_init_kernel(unsigned int* q_seq, unsigned int q_cap, unsigned int* ctr,
                                                      int n_ctr) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < q_cap) q_seq[i] = i;
    if (i < (unsigned)n_ctr) ctr[i] = 0u;
}

template <int L>
static cudaError_t kp_one(const KPParams& p, cudaStream_t st) {
    constexpr int LOGL = Sched<L, 32>::LOGL;
    static_assert(KNGeom<float, L>::G == KN_TILE_ROWS(LOGL) && KNGeom<float, L>::NT == KN_THREADS(LOGL),
                  "host-side task sizes follow the tile geometry");
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KNGeom<float, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kp_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(kp_kernel<L>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    if (ea != cudaSuccess) return ea;
    // one resident wave of CTAs
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp_kernel<L>, Gm::NT, Gm::smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kp_kernel<L><<<(unsigned)(sms * per_sm), Gm::NT, Gm::smem_bytes, st>>>(p);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t kp_launch(int logL, const KPParams& p, cudaStream_t st) {
    switch (logL) {
        case 8: return kp_one<256>(p, st);
        case 9: return kp_one<512>(p, st);
        case 10: return kp_one<1024>(p, st);
        case 11: return kp_one<2048>(p, st);
        case 12: return kp_one<4096>(p, st);
        case 13: return kp_one<8192>(p, st);
        case 14: return kp_one<16384>(p, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t kp_init_launch(unsigned int* q_seq, unsigned int q_cap, unsigned int* ctr, int n_ctr, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    const unsigned n = q_cap > (unsigned)n_ctr ? q_cap : (unsigned)n_ctr;
    kp_init_kernel<<<(n + 255) / 256, 256, 0, st>>>(q_seq, q_cap, ctr, n_ctr);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mpa
