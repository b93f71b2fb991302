// Launchers of the reverse-mode kernels, instantiated per precision by
// adj_f32.cu and adj_f64.cu.
#pragma once

#include "adj_launch.h"

namespace mpa {
namespace adj {

template <typename T, int L, int MODE>
cudaError_t kca_one(const KCAParams<T>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KCGeom<T, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kca_kernel<T, L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    if (p.ncols % Gm::G != 0) return cudaErrorInvalidValue;
    const long long nblk = p.ncols / Gm::G;
    if (nblk <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kca_kernel<T, L, MODE><<<(unsigned)nblk, Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) {
        // g read and written, plus one read of V_j or psi_j (a shared psi_0 once)
        const double cs = (double)sizeof(cx<T>), tile = (double)p.ncols * L;
        const double aux = p.aux_stride == 0 ? (double)p.N : tile;
        prof_end(PK_KC_ADJ, st, (2.0 * tile + aux) * cs);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T, int L>
cudaError_t kca_mode(int mode, const KCAParams<T>& p, cudaStream_t st) {
    return mode == KCA_G ? kca_one<T, L, KCA_G>(p, st) : kca_one<T, L, KCA_P>(p, st);
}

template <typename T, int L>
cudaError_t kra_one(const KRAParams<T>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KRGeom<T, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kra_kernel<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    if (p.nrows % Gm::G != 0) return cudaErrorInvalidValue;
    const long long nblk = p.nrows / Gm::G;
    if (nblk <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kra_kernel<T, L><<<(unsigned)nblk, Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) prof_end(PK_KR_ADJ, st, 3.0 * (double)p.nrows * L * sizeof(cx<T>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// The forward row pass of the recompute, keeping A(t) (KR_MPA_KEEP).
template <typename T, int L>
cudaError_t krk_one(const KRParams<T>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KRGeom<T, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kr_kernel<T, L, KR_MPA_KEEP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kr_kernel<T, L, KR_MPA_KEEP>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    if (!p.keep) return cudaErrorInvalidValue;
    const long long nblk = (p.nrows + Gm::G - 1) / Gm::G;
    if (nblk <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kr_kernel<T, L, KR_MPA_KEEP><<<(unsigned)nblk, Gm::NT, Gm::smem_bytes, st>>>(p);
    // rows read and written, A(t) written
    if (prof) prof_end(PK_KR_MPA, st, 3.0 * (double)p.nrows * L * sizeof(cx<T>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t krk_any(int logL, const KRParams<T>& p, cudaStream_t st) {
    switch (logL) {
        case 4: return krk_one<T, 16>(p, st);
        case 5: return krk_one<T, 32>(p, st);
        case 6: return krk_one<T, 64>(p, st);
        case 7: return krk_one<T, 128>(p, st);
        case 8: return krk_one<T, 256>(p, st);
        case 9: return krk_one<T, 512>(p, st);
        case 10: return krk_one<T, 1024>(p, st);
        case 11: return krk_one<T, 2048>(p, st);
        case 12: return krk_one<T, 4096>(p, st);
        case 13: return krk_one<T, 8192>(p, st);
        case 14:
            if constexpr (sizeof(T) == 4) return krk_one<T, 16384>(p, st);
            break;
    }
    return cudaErrorInvalidValue;
}

template <typename T, int L, int MODE>
cudaError_t ssc_one(const SSCParams<T>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KCGeom<T, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(ssc_kernel<T, L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    if (p.N1 % Gm::G != 0) return cudaErrorInvalidValue;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    ssc_kernel<T, L, MODE><<<(unsigned)(p.N1 / Gm::G), Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) prof_end(PK_KC_ADJ, st, 3.0 * (double)p.N * sizeof(cx<T>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T, int L, int MODE>
cudaError_t ssr_one(const SSRParams<T>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KRGeom<T, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(ssr_kernel<T, L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    if (p.nrows % Gm::G != 0) return cudaErrorInvalidValue;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    ssr_kernel<T, L, MODE><<<(unsigned)(p.nrows / Gm::G), Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) prof_end(PK_KR_ADJ, st, 3.0 * (double)p.nrows * L * sizeof(cx<T>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T, int L>
cudaError_t ssc_mode(int mode, const SSCParams<T>& p, cudaStream_t st) {
    return mode == SS_STORE ? ssc_one<T, L, SS_STORE>(p, st) : ssc_one<T, L, SS_REV>(p, st);
}
template <typename T, int L>
cudaError_t ssr_mode(int mode, const SSRParams<T>& p, cudaStream_t st) {
    return mode == SS_STORE ? ssr_one<T, L, SS_STORE>(p, st) : ssr_one<T, L, SS_REV>(p, st);
}

template <typename T>
cudaError_t ssc_any(int mode, int logL, const SSCParams<T>& p, cudaStream_t st) {
    switch (logL) {
        case 4: return ssc_mode<T, 16>(mode, p, st);
        case 5: return ssc_mode<T, 32>(mode, p, st);
        case 6: return ssc_mode<T, 64>(mode, p, st);
        case 7: return ssc_mode<T, 128>(mode, p, st);
        case 8: return ssc_mode<T, 256>(mode, p, st);
        case 9: return ssc_mode<T, 512>(mode, p, st);
        case 10: return ssc_mode<T, 1024>(mode, p, st);
        case 11: return ssc_mode<T, 2048>(mode, p, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t ssr_any(int mode, int logL, const SSRParams<T>& p, cudaStream_t st) {
    switch (logL) {
        case 4: return ssr_mode<T, 16>(mode, p, st);
        case 5: return ssr_mode<T, 32>(mode, p, st);
        case 6: return ssr_mode<T, 64>(mode, p, st);
        case 7: return ssr_mode<T, 128>(mode, p, st);
        case 8: return ssr_mode<T, 256>(mode, p, st);
        case 9: return ssr_mode<T, 512>(mode, p, st);
        case 10: return ssr_mode<T, 1024>(mode, p, st);
        case 11: return ssr_mode<T, 2048>(mode, p, st);
        case 12: return ssr_mode<T, 4096>(mode, p, st);
        case 13: return ssr_mode<T, 8192>(mode, p, st);
        case 14:
            if constexpr (sizeof(T) == 4) return ssr_mode<T, 16384>(mode, p, st);
            break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t kca_any(int mode, int logL, const KCAParams<T>& p, cudaStream_t st) {
    switch (logL) {
        case 4: return kca_mode<T, 16>(mode, p, st);
        case 5: return kca_mode<T, 32>(mode, p, st);
        case 6: return kca_mode<T, 64>(mode, p, st);
        case 7: return kca_mode<T, 128>(mode, p, st);
        case 8: return kca_mode<T, 256>(mode, p, st);
        case 9: return kca_mode<T, 512>(mode, p, st);
        case 10: return kca_mode<T, 1024>(mode, p, st);
        case 11: return kca_mode<T, 2048>(mode, p, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t kra_any(int logL, const KRAParams<T>& p, cudaStream_t st) {
    switch (logL) {
        case 4: return kra_one<T, 16>(p, st);
        case 5: return kra_one<T, 32>(p, st);
        case 6: return kra_one<T, 64>(p, st);
        case 7: return kra_one<T, 128>(p, st);
        case 8: return kra_one<T, 256>(p, st);
        case 9: return kra_one<T, 512>(p, st);
        case 10: return kra_one<T, 1024>(p, st);
        case 11: return kra_one<T, 2048>(p, st);
        case 12: return kra_one<T, 4096>(p, st);
        case 13: return kra_one<T, 8192>(p, st);
        case 14:
            if constexpr (sizeof(T) == 4) return kra_one<T, 16384>(p, st);
            break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
int kca_cols(int logL) {
    switch (logL) {
        case 4: return KCGeom<T, 16>::G;
        case 5: return KCGeom<T, 32>::G;
        case 6: return KCGeom<T, 64>::G;
        case 7: return KCGeom<T, 128>::G;
        case 8: return KCGeom<T, 256>::G;
        case 9: return KCGeom<T, 512>::G;
        case 10: return KCGeom<T, 1024>::G;
        case 11: return KCGeom<T, 2048>::G;
    }
    return -1;
}

template <typename T>
int kra_rows(int logL) {
    switch (logL) {
        case 4: return KRGeom<T, 16>::G;
        case 5: return KRGeom<T, 32>::G;
        case 6: return KRGeom<T, 64>::G;
        case 7: return KRGeom<T, 128>::G;
        case 8: return KRGeom<T, 256>::G;
        case 9: return KRGeom<T, 512>::G;
        case 10: return KRGeom<T, 1024>::G;
        case 11: return KRGeom<T, 2048>::G;
        case 12: return KRGeom<T, 4096>::G;
        case 13: return KRGeom<T, 8192>::G;
        case 14: return sizeof(T) == 4 ? KRGeom<T, 16384>::G : -1;
    }
    return -1;
}

template <typename T>
cudaError_t rscan_any(const RScanParams<T>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    const unsigned nb = (unsigned)((p.N + 255) / 256);
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    rscan_kernel<T><<<nb, 256, 0, st>>>(p);
    if (prof) {
        const double cs = (double)sizeof(cx<T>), nm = (double)(p.M + 1) * (double)p.N;
        const double b = p.mode == RSCAN_TOP ? nm * cs + 4.0 * 16.0 * p.N
                         : p.mode == RSCAN_LEVEL ? 2.0 * nm * cs + 32.0 * p.N
                                                 : nm * cs + 32.0 * p.N;
        prof_end(PK_ADJ_AUX, st, b);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t scan_store_any(const cx<T>* v, cx<T>* psi, const cx<T>* psi0c, long long N, int M, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    scan_store_kernel<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(v, psi, psi0c, N, M);
    if (prof) prof_end(PK_SCAN, st, (2.0 * (M + 1) + 1.0) * (double)N * sizeof(cx<T>));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t scale_to_state_any(const cx<T>* in, double2* state, double scale, long long N, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    scale_to_state_kernel<T><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(in, state, scale, N);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace adj
}  // namespace mpa

#define MPA_ADJ_INSTANTIATE_MPA(T)                                                                             \
    namespace mpa {                                                                                            \
    template <> cudaError_t kca_launch<T>(int mode, int logL, const KCAParams<T>& p, cudaStream_t st) {        \
        return adj::kca_any<T>(mode, logL, p, st);                                                             \
    }                                                                                                          \
    template <> cudaError_t kra_launch<T>(int logL, const KRAParams<T>& p, cudaStream_t st) {                  \
        return adj::kra_any<T>(logL, p, st);                                                                   \
    }                                                                                                          \
    template <> cudaError_t kr_keep_launch<T>(int logL, const KRParams<T>& p, cudaStream_t st) {               \
        return adj::krk_any<T>(logL, p, st);                                                                   \
    }                                                                                                          \
    template <> cudaError_t rscan_launch<T>(const RScanParams<T>& p, cudaStream_t st) {                        \
        return adj::rscan_any<T>(p, st);                                                                       \
    }                                                                                                          \
    template <>                                                                                                \
    cudaError_t scan_store_launch<T>(const cx<T>* v, cx<T>* psi, const cx<T>* psi0c, long long N, int M,      \
                                     cudaStream_t st) {                                                        \
        return adj::scan_store_any<T>(v, psi, psi0c, N, M, st);                                                \
    }                                                                                                          \
    template <>                                                                                                \
    cudaError_t scale_to_state_launch<T>(const cx<T>* in, double2* state, double scale, long long N,          \
                                         cudaStream_t st) {                                                    \
        return adj::scale_to_state_any<T>(in, state, scale, N, st);                                            \
    }                                                                                                          \
    template <> int kca_tile_cols<T>(int logL) { return adj::kca_cols<T>(logL); }                              \
    template <> int kra_tile_rows<T>(int logL) { return adj::kra_rows<T>(logL); }                              \
    }

#define MPA_ADJ_INSTANTIATE_SS(T)                                                                              \
    namespace mpa {                                                                                            \
    template <> cudaError_t ssc_launch<T>(int mode, int logL, const SSCParams<T>& p, cudaStream_t st) {        \
        return adj::ssc_any<T>(mode, logL, p, st);                                                             \
    }                                                                                                          \
    template <> cudaError_t ssr_launch<T>(int mode, int logL, const SSRParams<T>& p, cudaStream_t st) {        \
        return adj::ssr_any<T>(mode, logL, p, st);                                                             \
    }                                                                                                          \
    }
