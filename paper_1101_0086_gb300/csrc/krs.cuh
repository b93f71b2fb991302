// Staged, persistent row pass (FP32; MPA steps 3-4, or the split-step
// nonlinear step): the arithmetic of kr_kernel (inverse row DFTs, 1/N, the
// pointwise step, forward row DFTs, outer factor W_N^{+n2 k1}) on a schedule
// that overlaps each tile's HBM traffic with another tile's transforms.
//
// One CTA per SM holds two groups of NT threads.  The CTA's tiles are
// t_i = blockIdx.x + i gridDim.x (i = 0, 1, ...), and tile i goes to group
// i mod 2.  A tile's rows are contiguous in HBM; they arrive in a staging
// buffer that the two groups share, by bulk asynchronous copies
// (cp.async.bulk) whose bytes complete a phase of the receiving group's
// mbarrier.  A group waits for its tile, copies it from the stage into
// registers, and once all of its threads have done so (named barrier) and
// the first transform pass has moved the data on into the group's exchange
// buffer, one of them starts the copy of tile i + 1 (the other group's)
// into the stage.
// Each group transforms in its own exchange buffer with its own named
// barrier, so the next tile streams in and the two groups' transforms
// interleave on the SM while results go straight from registers to HBM.
//
// Group g's k-th tile completes phase k of mbarrier g; copy i + 1 is only
// started after tile i left the stage, so a barrier is never more than one
// phase ahead of its waiting group and parity waits are exact.  Every wait
// is bounded (spin_limit polls of mbarrier.try_wait): a wait that runs out
// sets ERR_TIMEOUT in the error word and the group stops; before a thread
// that started copies returns it waits (again bounded) for the last of them.
#pragma once

#include "kernels.cuh"

namespace mpa {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the asynchronous copy unit
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) whose bytes count against barrier b's transaction count
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(b))
                 : "memory");
}
// orders this thread's view of earlier shared-memory accesses (made visible
// to it by a barrier) before its later asynchronous-proxy copies
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Named barrier of the thread's NT-thread group that also returns whether
// any of the group's threads passed v = true.
template <int NT> __device__ __forceinline__ bool gsync_any(bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred q, p;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "r"(1 + (int)(threadIdx.x / NT)), "n"(NT)
        : "memory");
    return r != 0;
}

constexpr long long KRS_DRAIN_POLLS = 1ll << 24;

// Tile of the staged row pass: kr_kernel's G rows of L (8192 elements, 32
// per thread), with the outer factor W_N^{n2 k1} split at k1 = 32 h + m
// (kr_kernel splits at 128): tables of G (32 + L/32) entries per tile
// instead of G (128 + L/128), built per tile, and one low-table lookup per
// butterfly of the last radix-32 pass.
template <int L> struct KRSTile {
    typedef KRGeom<float, L> K;
    static constexpr int G = K::G, TE = K::TE, NT = K::NT;
    static constexpr int OSH = 5, OLO = L < 32 ? L : 32, OHI = L > 32 ? L / 32 : 1;
};

// Shared-memory layout of the staged row pass for row length L: the stage
// (TE elements), two mbarriers, the twiddle tables shared by both groups,
// then per group its exchange buffer and outer-factor tables.
template <int L> struct KRSGeom {
    typedef KRSTile<L> Gm;
    typedef Tiling<float, 1> P;
    static constexpr size_t al(size_t x) { return (x + 127) & ~(size_t)127; }
    static constexpr size_t STAGE_BYTES = (size_t)Gm::TE * sizeof(float2);
    static constexpr size_t BAR_OFF = STAGE_BYTES;
    static constexpr size_t TW_OFF = BAR_OFF + 128;
    static constexpr size_t GRP_OFF = al(TW_OFF + (size_t)(TwDims<L>::NLO + TwDims<L>::NHI) * sizeof(float2));
    static constexpr size_t S_ELEMS = (size_t)Gm::TE + (Gm::TE >> P::PSH) + 1;
    static constexpr size_t GRP_BYTES = al((S_ELEMS + (size_t)Gm::G * (Gm::OLO + Gm::OHI)) * sizeof(float2));
    static constexpr size_t smem_bytes = GRP_OFF + 2 * GRP_BYTES;
    static constexpr int NT = Gm::NT, THREADS = 2 * Gm::NT;
};

// Starts the copy of tile t's rows into the stage, counted on barrier b.
template <int L>
__device__ __forceinline__ void krs_fetch(const KRParams<float>& p, int t, float2* stage, unsigned long long* b) {
    constexpr int G = KRGeom<float, L>::G;
    const long long row0 = (long long)t * G;
    const long long nr = p.nrows - row0 < G ? p.nrows - row0 : G;
    const unsigned bytes = (unsigned)(nr * L * (long long)sizeof(float2));
    const char* src = reinterpret_cast<const char*>(p.data + row0 * L);
    if (!MPA_DBG_OK(p.dbg, src, bytes)) {
        mbar_arrive(b);  // debug build, range check failed: complete the phase without copying
        return;
    }
    mbar_arrive_expect_tx(b, bytes);
    char* dst = reinterpret_cast<char*>(stage);
    constexpr unsigned CH = 16384;
    for (unsigned o = 0; o < bytes; o += CH) bulk_g2s(dst + o, src + o, bytes - o < CH ? bytes - o : CH, b);
}

template <int L, int MODE>
__global__ void __launch_bounds__(KRSGeom<L>::THREADS, 1) krs_kernel(const KRParams<float> p, long long spin_limit) {
    static_assert(MODE == KR_MPA || MODE == KR_SS, "inverse, pointwise step and forward");
    typedef float2 C;
    typedef KRSTile<L> Gm;
    typedef KRSGeom<L> SG;
    typedef Tiling<float, 1> P;
    constexpr int G = Gm::G, NT = Gm::NT;
    typedef Xform<float, L, G, NT, P::RMAX, -1, LAYOUT_ROW, P::PSH, false, 1> XI;
    typedef Xform<float, L, G, NT, P::RMAX, +1, LAYOUT_ROW, P::PSH, true, 1> XF;
    static_assert(XI::RL == XF::R0, "inverse/forward junction radix");
    extern __shared__ __align__(128) unsigned char smem_staged[];
    C* stage = reinterpret_cast<C*>(smem_staged);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_staged + SG::BAR_OFF);
    C* thi = reinterpret_cast<C*>(smem_staged + SG::TW_OFF);
    C* tlo = thi + TwDims<L>::NHI;
    const int grp = (int)(threadIdx.x / NT), tid = (int)(threadIdx.x & (NT - 1));
    C* s = reinterpret_cast<C*>(smem_staged + SG::GRP_OFF + (size_t)grp * SG::GRP_BYTES);
    C* olo = s + SG::S_ELEMS;   // [G][OLO]
    C* ohi = olo + G * Gm::OLO; // [G][OHI]
    const int ntiles = (int)((p.nrows + G - 1) / G);  // < 2^31: rows of a launch / G

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    tw_init<float, L>(thi, tlo, (int)threadIdx.x, SG::THREADS);
    __syncthreads();
    int last_copy = -1;  // CTA-local index of the last tile this thread started copying
    if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) {
        krs_fetch<L>(p, blockIdx.x, stage, &bar[0]);
        last_copy = 0;
    }

    unsigned k = 0;            // the group's tile count = its barrier's phase
    for (int i = grp;; i += 2, ++k) {
        const int t = (int)blockIdx.x + i * (int)gridDim.x;
        if (t >= ntiles) break;
        const long long row0 = (long long)t * G;
        gsync<1, NT>();  // the group's previous tile no longer needs s, olo, ohi
        // W_N^{+n2 k1} for the tile's rows: olo[g][m] = W^{n2 m}, ohi[g][h] = W^{n2 32 h}
        for (int e = tid; e < G * (Gm::OLO + Gm::OHI); e += NT) {
            const int g = e / (Gm::OLO + Gm::OHI), m = e % (Gm::OLO + Gm::OHI);
            const long long n2 = (row0 + g) & (p.N2 - 1);
            if (m < Gm::OLO) olo[g * Gm::OLO + m] = expi_ratio<float>(n2 * m, p.logN);
            else ohi[g * Gm::OHI + (m - Gm::OLO)] = expi_ratio<float>(n2 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
        }
        bool ok = false;
        for (long long w = 0; w < spin_limit && !ok; ++w) ok = mbar_try_wait(&bar[grp], k & 1u);
        C vin[XI::Q0][XI::R0];
#pragma unroll
        for (int q = 0; q < XI::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_ROW, L, G, XI::R0>(tid + q * NT, j, g);
            const bool in = ok && row0 + g < p.nrows;
            const C* src = stage + g * L;
#pragma unroll
            for (int r = 0; r < XI::R0; ++r) vin[q][r] = in ? src[j + r * (L / XI::R0)] : mkc(0.f, 0.f);
        }
        // every thread of the group has its part of the tile (and the tables are written)
        if (gsync_any<NT>(!ok)) {
            if (tid == 0) atomicOr(p.err, ERR_TIMEOUT);
            break;
        }
        C vm[XI::QL][XI::RL];
        // the next tile's copy starts once the first pass has left the registers
        XI::run(vin, vm, s, thi, tlo, [&] {
            const int tn = t + (int)gridDim.x;
            if (tid == 0 && tn < ntiles) {
                fence_proxy_async_smem();
                krs_fetch<L>(p, tn, stage, &bar[grp ^ 1]);
                last_copy = i + 1;
            }
        });
#pragma unroll
        for (int q = 0; q < XI::QL; ++q) {
#pragma unroll
            for (int r = 0; r < XI::RL; ++r) {
                C a = cscale(vm[q][r], p.inv_n);  // A(t) (MPA step 3 / SS inverse)
                const float pw = a.x * a.x + a.y * a.y;
                if constexpr (MODE == KR_MPA) {
                    a = cscale(a, pw);  // |A|^2 A (MPA step 4)
                } else {
                    float sn, cs;  // A exp(i s |A|^2), the nonlinear step of Eq. (4)
                    sincos_kerr(p.rot * pw, &sn, &cs);
                    a = cmul(a, mkc(cs, sn));
                }
                vm[q][r] = a;
            }
        }
        C vout[XF::QL][XF::RL];
        XF::run(vm, vout, s, thi, tlo);
#pragma unroll
        for (int q = 0; q < XF::QL; ++q) {
            int j, g;
            bmap<LAYOUT_ROW, L, G, XF::RL>(tid + q * NT, j, g);
            if (row0 + g >= p.nrows) continue;
            C* dst = p.data + (row0 + g) * L;
            constexpr bool HOIST = (L / XF::RL) % Gm::OLO == 0;  // one low-table lookup per butterfly
            C wlo = mkc(1.f, 0.f);
            if constexpr (HOIST) wlo = olo[g * Gm::OLO + (j & (Gm::OLO - 1))];
#pragma unroll
            for (int r = 0; r < XF::RL; ++r) {
                const int l = j + r * (L / XF::RL);  // k1
                C w = HOIST ? wlo : olo[g * Gm::OLO + (l & (Gm::OLO - 1))];
                if constexpr (Gm::OHI > 1) w = cmul(ohi[g * Gm::OHI + (l >> Gm::OSH)], w);
                if (MPA_DBG_OK(p.dbg, dst + l, sizeof(C))) dst[l] = cmul(vout[q][r], w);
            }
        }
    }
    // the block's shared memory must outlive the last copy this thread
    // started (only copies a group abandoned after a timeout can still be in
    // flight here; a copy lands within microseconds, so this limit is only a
    // bound and independent of spin_limit)
    if (last_copy >= 0) {
        const int gb = (int)(last_copy & 1);
        const unsigned kb = (unsigned)(last_copy >> 1);
        bool done = false;
        for (long long w = 0; w < KRS_DRAIN_POLLS && !done; ++w) done = mbar_try_wait(&bar[gb], kb & 1u);
        if (!done) atomicOr(p.err, ERR_TIMEOUT);
    }
}

}  // namespace mpa
