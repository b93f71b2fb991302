// Launchers of the on-chip whole node transform, float.
#include "launch.h"

namespace mpa {

template <int L>
static cudaError_t kn_one(const KNParams<float>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KNGeom<float, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kn_kernel<float, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(kn_kernel<float, L>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    });
    if (ea != cudaSuccess) return ea;
    const long long nblk = (p.nrows + Gm::G - 1) / Gm::G;
    if (nblk <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kn_kernel<float, L><<<(unsigned)nblk, Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) {
        // every node read once and written once (a shared psi_0 once per link)
        const double cs = (double)sizeof(cx<float>), nodes = (double)p.nrows;
        const double rd = p.src_stride == 0 ? nodes / p.npl : nodes;
        prof_end(PK_KN, st, (rd + nodes) * L * cs);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <>
cudaError_t kn_launch<float>(int logL, const KNParams<float>& p, cudaStream_t st) {
    switch (logL) {
        case 8: return kn_one<256>(p, st);
        case 9: return kn_one<512>(p, st);
        case 10: return kn_one<1024>(p, st);
        case 11: return kn_one<2048>(p, st);
        case 12: return kn_one<4096>(p, st);
        case 13: return kn_one<8192>(p, st);
        case 14: return kn_one<16384>(p, st);
        case 15:
        case 16: return knc_launch(logL, p, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mpa
