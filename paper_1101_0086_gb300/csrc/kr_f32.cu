// Row-pass launchers, float.
#include "krs.cuh"
#include "launch.h"

namespace mpa {

// The staged persistent row pass (krs.cuh) for rows of 2^9 .. 2^13 points
// in the MPA and split-step modes, whenever the caller passes an error word
// for its bounded waits; MPA_KR_STAGED=0 keeps kr_kernel everywhere.
#ifndef MPA_KR_STAGED
#define MPA_KR_STAGED 1
#endif

template <int L, int MODE>
static cudaError_t krs_one(const KRParams<float>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KRSGeom<L> SG;
    static_assert(SG::smem_bytes <= 227u * 1024u, "staged row pass exceeds the shared memory of an SM");
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        return cudaFuncSetAttribute(krs_kernel<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SG::smem_bytes);
    });
    if (ea != cudaSuccess) return ea;
    const long long ntiles = (p.nrows + KRGeom<float, L>::G - 1) / KRGeom<float, L>::G;
    if (ntiles <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);  // one CTA per SM
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    krs_kernel<L, MODE><<<grid, SG::THREADS, SG::smem_bytes, st>>>(p, p.spin_limit);
    if (prof) prof_end(prof_kr_kind(MODE), st, 2.0 * (double)p.nrows * L * sizeof(cx<float>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <int L>
static cudaError_t krs_mode(int mode, const KRParams<float>& p, cudaStream_t st) {
    return mode == KR_MPA ? krs_one<L, KR_MPA>(p, st) : krs_one<L, KR_SS>(p, st);
}

bool kr_staged(int mode, int logL, const KRParams<float>& p) {
    return MPA_KR_STAGED && p.err && (mode == KR_MPA || mode == KR_SS) && logL >= 9 && logL <= 13;
}

template <int L, int MODE>
static cudaError_t kr_one(const KRParams<float>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KRGeom<float, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kr_kernel<float, L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kr_kernel<float, L, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    const long long nblk = (p.nrows + Gm::G - 1) / Gm::G;
    if (nblk <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kr_kernel<float, L, MODE><<<(unsigned)nblk, Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) prof_end(prof_kr_kind(MODE), st, 2.0 * (double)p.nrows * L * sizeof(cx<float>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <int L>
static cudaError_t kr_mode(int mode, const KRParams<float>& p, cudaStream_t st) {
    switch (mode) {
        case KR_MPA: return kr_one<L, KR_MPA>(p, st);
        case KR_SS: return kr_one<L, KR_SS>(p, st);
        case KR_FWD: return kr_one<L, KR_FWD>(p, st);
        case KR_INV: return kr_one<L, KR_INV>(p, st);
    }
    return cudaErrorInvalidValue;
}

template <>
cudaError_t kr_launch<float>(int mode, int logL, const KRParams<float>& p, cudaStream_t st) {
    if (kr_staged(mode, logL, p)) {
        switch (logL) {
            case 9: return krs_mode<512>(mode, p, st);
            case 10: return krs_mode<1024>(mode, p, st);
            case 11: return krs_mode<2048>(mode, p, st);
            case 12: return krs_mode<4096>(mode, p, st);
            case 13: return krs_mode<8192>(mode, p, st);
        }
    }
    switch (logL) {
        case 4: return kr_mode<16>(mode, p, st);
        case 5: return kr_mode<32>(mode, p, st);
        case 6: return kr_mode<64>(mode, p, st);
        case 7: return kr_mode<128>(mode, p, st);
        case 8: return kr_mode<256>(mode, p, st);
        case 9: return kr_mode<512>(mode, p, st);
        case 10: return kr_mode<1024>(mode, p, st);
        case 11: return kr_mode<2048>(mode, p, st);
        case 12: return kr_mode<4096>(mode, p, st);
        case 13: return kr_mode<8192>(mode, p, st);
        case 14: return kr_mode<16384>(mode, p, st);
    }
    return cudaErrorInvalidValue;
}

template <>
long long kr_blocks<float>(int logL, long long nrows) {
    switch (logL) {
        case 4: return (nrows + KRGeom<float, 16>::G - 1) / KRGeom<float, 16>::G;
        case 5: return (nrows + KRGeom<float, 32>::G - 1) / KRGeom<float, 32>::G;
        case 6: return (nrows + KRGeom<float, 64>::G - 1) / KRGeom<float, 64>::G;
        case 7: return (nrows + KRGeom<float, 128>::G - 1) / KRGeom<float, 128>::G;
        case 8: return (nrows + KRGeom<float, 256>::G - 1) / KRGeom<float, 256>::G;
        case 9: return (nrows + KRGeom<float, 512>::G - 1) / KRGeom<float, 512>::G;
        case 10: return (nrows + KRGeom<float, 1024>::G - 1) / KRGeom<float, 1024>::G;
        case 11: return (nrows + KRGeom<float, 2048>::G - 1) / KRGeom<float, 2048>::G;
        case 12: return (nrows + KRGeom<float, 4096>::G - 1) / KRGeom<float, 4096>::G;
        case 13: return (nrows + KRGeom<float, 8192>::G - 1) / KRGeom<float, 8192>::G;
        case 14: return (nrows + KRGeom<float, 16384>::G - 1) / KRGeom<float, 16384>::G;
    }
    return -1;
}

}  // namespace mpa
