// Column-pass launchers, float.
#include "kcs.cuh"
#include "launch.h"

namespace mpa {

// The staged persistent column pass (kcs.cuh) for the MPA passes with
// columns of 2^8 .. 2^11 points and tiles within one node (N1 a multiple of
// the tile width), whenever the caller passes an error word for its bounded
// waits; MPA_KC_STAGED=0 keeps kc_kernel everywhere.
#ifndef MPA_KC_STAGED
#define MPA_KC_STAGED 1
#endif

template <int L, int MODE>
static cudaError_t kcs_one(const KCParams<float>& p, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KCSGeom<L> SG;
    static_assert(SG::smem_bytes <= 227u * 1024u, "staged column pass exceeds the shared memory of an SM");
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        return cudaFuncSetAttribute(kcs_kernel<L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SG::smem_bytes);
    });
    if (ea != cudaSuccess) return ea;
    const long long ntiles = p.ncols / KCSTile<L>::G;
    if (ntiles <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);  // one CTA per SM
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kcs_kernel<L, MODE><<<grid, SG::THREADS, SG::smem_bytes, st>>>(p);
    if (prof) {
        const double cs = (double)sizeof(cx<float>), tile = (double)p.ncols * L;
        const double rd = p.src_stride == 0 ? (double)p.ncols / p.npl * L : tile;
        prof_end(prof_kc_kind(MODE), st, (rd + tile) * cs);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

static constexpr int ilog2_const(int x) { return x <= 1 ? 0 : 1 + ilog2_const(x / 2); }

template <int L> static bool kcs_fits(const KCParams<float>& p) {
    return p.N1 % KCSTile<L>::G == 0 && p.ncols % KCSTile<L>::G == 0;
}

bool kc_staged(int mode, int logL, const KCParams<float>& p) {
    if (!MPA_KC_STAGED || !p.err || (mode != KC_MPA_PRE && mode != KC_MPA_POST) || p.npl <= 0) return false;
    switch (logL) {
        case 8: return kcs_fits<256>(p);
        case 9: return kcs_fits<512>(p);
        case 10: return kcs_fits<1024>(p);
        case 11: return kcs_fits<2048>(p);
    }
    return false;
}

int kcs_tile_log_cols(int logL) {
    switch (logL) {
        case 8: return ilog2_const(KCSTile<256>::G);
        case 9: return ilog2_const(KCSTile<512>::G);
        case 10: return ilog2_const(KCSTile<1024>::G);
        case 11: return ilog2_const(KCSTile<2048>::G);
    }
    return -1;
}

template <int L> static cudaError_t kcs_mode(int mode, const KCParams<float>& p, cudaStream_t st) {
    return mode == KC_MPA_PRE ? kcs_one<L, KC_MPA_PRE>(p, st) : kcs_one<L, KC_MPA_POST>(p, st);
}

template <int L, int MODE>
static cudaError_t kc_one(const KCParams<float>& pin, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    // callers that leave the link fields unset launch one run of nodes
    KCParams<float> p = pin;
    if (p.npl <= 0) p.npl = (int)(p.ncols >> p.logN1) > 0 ? (int)(p.ncols >> p.logN1) : 1;
    typedef KCGeom<float, L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kc_kernel<float, L, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kc_kernel<float, L, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    const long long nblk = (p.ncols + Gm::G - 1) / Gm::G;
    if (nblk <= 0) return cudaSuccess;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kc_kernel<float, L, MODE><<<(unsigned)nblk, Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) {
        // algorithmic bytes: every tile element read once and written once
        // (a shared source, src_stride == 0, is read once for all nodes)
        const double cs = (double)sizeof(cx<float>), tile = (double)p.ncols * L;
        const double rd = p.src_stride == 0 ? (double)p.ncols / p.npl * L : tile;
        prof_end(prof_kc_kind(MODE), st, (rd + tile) * cs);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <int L>
static cudaError_t kc_mode(int mode, const KCParams<float>& p, cudaStream_t st) {
    switch (mode) {
        case KC_MPA_PRE: return kc_one<L, KC_MPA_PRE>(p, st);
        case KC_MPA_POST: return kc_one<L, KC_MPA_POST>(p, st);
        case KC_SS_STEP: return kc_one<L, KC_SS_STEP>(p, st);
        case KC_FWD: return kc_one<L, KC_FWD>(p, st);
        case KC_INV: return kc_one<L, KC_INV>(p, st);
    }
    return cudaErrorInvalidValue;
}

template <>
cudaError_t kc_launch<float>(int mode, int logL, const KCParams<float>& p, cudaStream_t st) {
    if (kc_staged(mode, logL, p)) {
        switch (logL) {
            case 8: return kcs_mode<256>(mode, p, st);
            case 9: return kcs_mode<512>(mode, p, st);
            case 10: return kcs_mode<1024>(mode, p, st);
            case 11: return kcs_mode<2048>(mode, p, st);
        }
    }
    switch (logL) {
        case 4: return kc_mode<16>(mode, p, st);
        case 5: return kc_mode<32>(mode, p, st);
        case 6: return kc_mode<64>(mode, p, st);
        case 7: return kc_mode<128>(mode, p, st);
        case 8: return kc_mode<256>(mode, p, st);
        case 9: return kc_mode<512>(mode, p, st);
        case 10: return kc_mode<1024>(mode, p, st);
        case 11: return kc_mode<2048>(mode, p, st);
    }
    return cudaErrorInvalidValue;
}

template <>
long long kc_blocks<float>(int logL, long long ncols) {
    switch (logL) {
        case 4: return (ncols + KCGeom<float, 16>::G - 1) / KCGeom<float, 16>::G;
        case 5: return (ncols + KCGeom<float, 32>::G - 1) / KCGeom<float, 32>::G;
        case 6: return (ncols + KCGeom<float, 64>::G - 1) / KCGeom<float, 64>::G;
        case 7: return (ncols + KCGeom<float, 128>::G - 1) / KCGeom<float, 128>::G;
        case 8: return (ncols + KCGeom<float, 256>::G - 1) / KCGeom<float, 256>::G;
        case 9: return (ncols + KCGeom<float, 512>::G - 1) / KCGeom<float, 512>::G;
        case 10: return (ncols + KCGeom<float, 1024>::G - 1) / KCGeom<float, 1024>::G;
        case 11: return (ncols + KCGeom<float, 2048>::G - 1) / KCGeom<float, 2048>::G;
    }
    return -1;
}

}  // namespace mpa
