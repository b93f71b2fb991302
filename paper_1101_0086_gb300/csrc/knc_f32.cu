// Launchers of the cluster on-chip node transform (FP32, N = 2^15, 2^16).
#include "knc.cuh"
#include "launch.h"

namespace mpa {

template <int C>
static cudaError_t knc_one(const KNParams<float>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KNCGeom<C> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        return cudaFuncSetAttribute(knc_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_bytes);
    });
    if (ea != cudaSuccess) return ea;
    if (p.nrows <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    knc_kernel<C><<<(unsigned)(p.nrows * C), Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) {
        const double cs = (double)sizeof(float2), nodes = (double)p.nrows, L = (double)C * Gm::P;
        const double rd = p.src_stride == 0 ? nodes / p.npl : nodes;
        prof_end(PK_KN, st, (rd + nodes) * L * cs);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t knc_launch(int logL, const KNParams<float>& p, cudaStream_t st) {
    switch (logL) {
        case 15: return knc_one<2>(p, st);
        case 16: return knc_one<4>(p, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mpa
