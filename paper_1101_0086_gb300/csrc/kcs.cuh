// Staged, persistent column pass (FP32; the MPA column passes): the
// arithmetic of kc_kernel in modes KC_MPA_PRE (phase exp(i beta_j + int G),
// inverse column DFTs, outer factor W_N^{-n2 k1}) and KC_MPA_POST (forward
// column DFTs, V_j of Eq. (6)) on the schedule of the staged row pass
// (krs.cuh): one CTA per SM, two groups of NT threads taking the CTA's
// tiles in turn, and one staging buffer that the next tile streams into
// while the current ones are transformed.
//
// A column tile is G columns x L rows of one node (the tile never straddles
// nodes: N1 is a multiple of G), i.e. L row segments of G complex64 (32 to
// 256 bytes for L = 2^11 .. 2^8) at a stride of N1 elements.  Such short strided segments are copied by the
// NT threads of the group that releases the stage, 16 bytes per cp.async
// (a bulk copy per segment was measured 2.3x slower: each bulk request has
// a fixed cost), and each thread arrives on the receiving group's mbarrier
// when its own copies have landed (cp.async.mbarrier.arrive.noinc; the
// barrier counts NT arrivals per phase).  Waits are bounded as in krs.cuh;
// every thread waits for its own copies before it returns.
#pragma once

#include "krs.cuh"

namespace mpa {

// Tile of the staged column pass: G = 8192 / L columns (at least 4) of L
// rows, 32 elements per thread; the per-tile kc_kernel keeps G >= 8, which
// makes 2^11-point column tiles 16384 elements, too large to stage.  The
// outer-factor split is kc_kernel's.
template <int L> struct KCSTile {
    typedef KCGeom<float, L> K;
    static constexpr int G = (8192 / L) > 4 ? (8192 / L) : 4, TE = G * L, NT = TE / Tiling<float>::E;
    static constexpr int OSH = K::OSH, OLO = K::OLO, OHI = K::OHI;
};

// Shared-memory layout: the stage (TE elements, row-major L x G), two
// mbarriers, four slots of node constants (those of CTA-local tile i in
// slot i mod 4, copied with the tile), the twiddle tables of both groups,
// then per group its exchange buffer and outer-factor tables.
template <int L> struct KCSGeom {
    typedef KCSTile<L> Gm;
    typedef Tiling<float> P;
    static constexpr size_t al(size_t x) { return (x + 127) & ~(size_t)127; }
    static constexpr size_t STAGE_BYTES = (size_t)Gm::TE * sizeof(float2);
    static constexpr size_t BAR_OFF = STAGE_BYTES;
    static constexpr size_t NODE_OFF = BAR_OFF + 16;  // 4 NodeC slots: tile i's node constants in slot i mod 4
    static constexpr size_t TW_OFF = BAR_OFF + 256;
    static_assert(sizeof(NodeC) == 48 && 16 + 4 * sizeof(NodeC) <= 256, "node-constant slots");
    static constexpr size_t GRP_OFF = al(TW_OFF + (size_t)(TwDims<L>::NLO + TwDims<L>::NHI) * sizeof(float2));
    static constexpr size_t S_ELEMS = (size_t)Gm::TE + (Gm::TE >> P::PSH) + 1;
    static constexpr size_t GRP_BYTES = al((S_ELEMS + (size_t)Gm::G * (Gm::OLO + Gm::OHI)) * sizeof(float2));
    static constexpr size_t smem_bytes = GRP_OFF + 2 * GRP_BYTES;
    static constexpr int NT = Gm::NT, THREADS = 2 * Gm::NT;
};

// Node and link of column col (the launch layout of kc_kernel), c its column
// within the node.
__host__ __device__ __forceinline__ void kcs_node(const KCParams<float>& p, long long col, int& l, int& jn, long long& c) {
    const int node = (int)(col >> p.logN1);
    l = node / p.npl;
    jn = node - l * p.npl;
    c = col & (long long)(p.N1 - 1);
}
// Where the tile of G columns starting at column c of (link l, node jn)
// begins and the distance between its rows, in elements: natural order
// (row stride N1) or the tile layout (the tile's G x L elements contiguous
// at c L, row stride G).
template <int L, int G>
__host__ __device__ __forceinline__ const float2* kcs_src(const KCParams<float>& p, int l, int jn, long long c,
                                                          long long& rs) {
    if (p.src0 && jn == 0) {
        rs = p.N1;
        return p.src0 + l * p.src0_lstride + c;
    }
    const float2* b = p.src + l * p.src_lstride + jn * p.src_stride;
    rs = p.tiled_in ? G : p.N1;
    return p.tiled_in ? b + c * L : b + c;
}
template <int L, int G>
__host__ __device__ __forceinline__ float2* kcs_dst(const KCParams<float>& p, int l, int jn, long long c, long long& rs) {
    float2* b = p.dst + l * p.dst_lstride + jn * p.dst_stride;
    rs = p.tiled_out ? G : p.N1;
    return p.tiled_out ? b + c * L : b + c;
}

// 16-byte global -> shared copy through L2 (cp.async.cg)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// barrier b receives one arrival from this thread once all of its earlier
// cp.async copies have landed (the arrival is counted in b's expected count)
__device__ __forceinline__ void cp_async_arrive(unsigned long long* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Group-wide: the NT threads start the copies of tile t (L row segments of
// G elements) into the stage, and three of them the copy of the tile's node
// constants into `slot`; each thread arrives on barrier b when its copies
// have landed.
template <int L>
__device__ __forceinline__ void kcs_fetch(const KCParams<float>& p, int t, float2* stage, NodeC* slot,
                                          unsigned long long* b, int tid) {
    constexpr int G = KCSTile<L>::G, NT = KCSTile<L>::NT;
    constexpr int CPR = G * (int)sizeof(float2) / 16;  // 16-byte chunks per row segment
    constexpr int NCH = L * CPR;
    static_assert(NCH % NT == 0, "whole chunks per thread");
    int l, jn;
    long long c, rs;
    kcs_node(p, (long long)t * G, l, jn, c);
    const char* src = reinterpret_cast<const char*>(kcs_src<L, G>(p, l, jn, c, rs));
    char* dst = reinterpret_cast<char*>(stage);
#pragma unroll
    for (int k = 0; k < NCH / NT; ++k) {
        const int id = tid + k * NT, row = id / CPR, ch = id % CPR;
        const char* from = src + (long long)row * rs * (long long)sizeof(float2) + ch * 16;
        if (MPA_DBG_OK(p.dbg, from, 16)) cp_async16(dst + (size_t)row * G * sizeof(float2) + ch * 16, from);
    }
    if (tid < (int)(sizeof(NodeC) / 16) && MPA_DBG_OK(p.dbg, p.loff + l, sizeof(int))) {
        const char* from = reinterpret_cast<const char*>(p.nodes + p.loff[l] + jn) + 16 * tid;
        if (MPA_DBG_OK(p.dbg, from, 16)) cp_async16(reinterpret_cast<char*>(slot) + 16 * tid, from);
    }
    cp_async_arrive(b);  // arrives once this thread's issued copies have landed (none: at once)
}

// Group-wide: asks L2 for tile t's row segments (cp.async.bulk.prefetch), so
// that the copies of the tile, started one tile later, find them there.
template <int L>
__device__ __forceinline__ void kcs_prefetch(const KCParams<float>& p, int t, int tid) {
    constexpr int G = KCSTile<L>::G, NT = KCSTile<L>::NT;
    int l, jn;
    long long c, rs;
    kcs_node(p, (long long)t * G, l, jn, c);
    const float2* src = kcs_src<L, G>(p, l, jn, c, rs);
    for (int row = tid; row < L; row += NT) prefetch_l2(src + (long long)row * rs, (unsigned)(G * sizeof(float2)));
}

// L2 prefetch of the tile after next in the staged column passes (bit 0:
// inverse pass, bit 1: forward pass).  Measured on the 2^20 link: slower in
// both passes (inverse 69 -> 81 ms, forward 54 -> 75 ms per 100 km at the
// 2^10 x 2^10 split), so off.
#ifndef MPA_KCS_L2PF
#define MPA_KCS_L2PF 0
#endif

template <int L, int MODE>
__global__ void __launch_bounds__(KCSGeom<L>::THREADS, 1)
    kcs_kernel(const KCParams<float> p) {
    static_assert(MODE == KC_MPA_PRE || MODE == KC_MPA_POST, "the MPA column passes");
    typedef float2 C;
    typedef KCSTile<L> Gm;
    typedef KCSGeom<L> SG;
    typedef Tiling<float> P;
    constexpr int G = Gm::G, NT = Gm::NT;
    constexpr bool INV = MODE == KC_MPA_PRE;
    typedef Xform<float, L, G, NT, P::RMAX, +1, LAYOUT_COL, P::PSH, true, 1> XF;
    typedef Xform<float, L, G, NT, P::RMAX, -1, LAYOUT_COL, P::PSH, false, 1> XI;
    typedef typename std::conditional<INV, XI, XF>::type XA;
    extern __shared__ __align__(128) unsigned char smem_staged[];
    C* stage = reinterpret_cast<C*>(smem_staged);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_staged + SG::BAR_OFF);
    NodeC* nslot = reinterpret_cast<NodeC*>(smem_staged + SG::NODE_OFF);
    C* thi = reinterpret_cast<C*>(smem_staged + SG::TW_OFF);
    C* tlo = thi + TwDims<L>::NHI;
    const int grp = (int)(threadIdx.x / NT), tid = (int)(threadIdx.x & (NT - 1));
    C* s = reinterpret_cast<C*>(smem_staged + SG::GRP_OFF + (size_t)grp * SG::GRP_BYTES);
    C* olo = s + SG::S_ELEMS;   // [OLO][G]
    C* ohi = olo + G * Gm::OLO; // [OHI][G]
    const int ntiles = (int)(p.ncols / G);  // < 2^31: columns of a launch / G
    const int N1m = p.N1 - 1;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], NT);
        mbar_init(&bar[1], NT);
        mbar_init_fence();
    }
    tw_init<float, L>(thi, tlo, (int)threadIdx.x, SG::THREADS);
    __syncthreads();
    // the first tile is copied by group 1 (whose own first tile comes later)
    if (grp == 1 && (int)blockIdx.x < ntiles) kcs_fetch<L>(p, blockIdx.x, stage, &nslot[0], &bar[0], tid);

    unsigned k = 0;
    for (int i = grp;; i += 2, ++k) {
        const int t = (int)blockIdx.x + i * (int)gridDim.x;
        if (t >= ntiles) break;
        const long long col0 = (long long)t * G;
        // the tile's link, node and first column within the node (a tile never straddles nodes)
        int tl, tjn;
        long long tc0;
        kcs_node(p, col0, tl, tjn, tc0);
        gsync<1, NT>();  // the group's previous tile no longer needs s, olo, ohi
        if constexpr (INV) {
            // W_N^{-n2 k1} for the tile's columns: olo[m][g] = W^{-k1 m}, ohi[h][g] = W^{-k1 32 h}
            for (int e = tid; e < G * (Gm::OLO + Gm::OHI); e += NT) {
                const int g = e % G, m = e / G;
                const long long k1 = (col0 + g) & N1m;
                if (m < Gm::OLO) olo[m * G + g] = expi_ratio<float>(-k1 * m, p.logN);
                else ohi[(m - Gm::OLO) * G + g] = expi_ratio<float>(-k1 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
            }
        }
        bool ok = false;
        for (long long w = 0; w < p.spin_limit && !ok; ++w) ok = mbar_try_wait(&bar[grp], k & 1u);

        // ---- element j + r L/R0 of column col0 + g, from the stage
        C vin[XA::Q0][XA::R0];
#pragma unroll
        for (int q = 0; q < XA::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, G, XA::R0>(tid + q * NT, j, g);
            if constexpr (INV) {
                const long long c = tc0 + g;
                const NodeC nc = nslot[i & 3];  // copied with the tile
                // phases in the order of their finite differences: s = -R0/2 .. R0/2-1,
                // element r = (s + R0) mod R0 at k' = c + N1 (j + s L/R0)
                const long long D = (long long)p.N1 * (L / XA::R0);
                PhaseRun pr(c + (long long)j * p.N1 - (long long)(XA::R0 / 2) * D, D, nc);
#pragma unroll
                for (int u = 0; u < XA::R0; ++u) {
                    const int r = (u + XA::R0 / 2) % XA::R0;
                    const int row = j + r * (L / XA::R0);
                    const C v = ok ? stage[row * G + g] : mkc(0.f, 0.f);
                    // MPA step 2: A_hat_j = psi_j exp(i beta(w, z_j) + int G)
                    vin[q][r] = cscale(cmul(v, expi_turns_poly(pr.next())), (float)nc.pre);
                }
            } else {
#pragma unroll
                for (int r = 0; r < XA::R0; ++r) {
                    const int row = j + r * (L / XA::R0);
                    vin[q][r] = ok ? stage[row * G + g] : mkc(0.f, 0.f);
                }
            }
        }
        // every thread of the group has its part of the tile (and the tables are written)
        if (gsync_any<NT>(!ok)) {
            if (tid == 0) atomicOr(p.err, ERR_TIMEOUT);
            break;
        }
        // The next tile's copies start here, or (LATE) once the first transform
        // pass has moved the tile out of the registers: the inverse pass of
        // 256- and 2048-point columns spills registers if they start here,
        // while the others lose time if they start later (the other group waits).
        constexpr bool LATE = INV && (L == 256 || L == 2048);
        auto fetch_next = [&] {
            const int tn = t + (int)gridDim.x;
            if (tn < ntiles) kcs_fetch<L>(p, tn, stage, &nslot[(i + 1) & 3], &bar[grp ^ 1], tid);
            constexpr bool PF = (MPA_KCS_L2PF >> (INV ? 0 : 1)) & 1;
            if constexpr (PF) {
                const int tp = tn + (int)gridDim.x;
                if (tp < ntiles) kcs_prefetch<L>(p, tp, tid);
            }
        };
        if constexpr (!LATE) fetch_next();
        constexpr int QO = XA::QL, RO = XA::RL;
        C vout[QO][RO];
        XA::run(vin, vout, s, thi, tlo, [&] {
            if constexpr (LATE) fetch_next();
        });

        // ---- epilogue and store: element j + r L/RO of column col0 + g
#pragma unroll
        for (int q = 0; q < QO; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, G, RO>(tid + q * NT, j, g);
            const long long c = tc0 + g;
            long long rs;
            // natural order, or the tile layout: the tile block at column tc0, element g
            C* dst = kcs_dst<L, G>(p, tl, tjn, tc0, rs) + g;
            if constexpr (INV) {
                constexpr bool HOIST = (L / RO) % Gm::OLO == 0;
                C wlo = mkc(1.f, 0.f);
                if constexpr (HOIST) wlo = olo[(j & (Gm::OLO - 1)) * G + g];
#pragma unroll
                for (int r = 0; r < RO; ++r) {
                    const int row = j + r * (L / RO);
                    // four-step factor W_N^{-n2 k1}, n2 = row
                    C w = HOIST ? wlo : olo[(row & (Gm::OLO - 1)) * G + g];
                    if constexpr (Gm::OHI > 1) w = cmul(ohi[(row >> Gm::OSH) * G + g], w);
                    if (MPA_DBG_OK(p.dbg, dst + (long long)row * rs, sizeof(C))) dst[(long long)row * rs] = cmul(vout[q][r], w);
                }
            } else {
                const NodeC nc = nslot[i & 3];  // copied with the tile
                const long long D = (long long)p.N1 * (L / RO);
                PhaseRun pr(c + (long long)j * p.N1 - (long long)(RO / 2) * D, D, nc);
#pragma unroll
                for (int u = 0; u < RO; ++u) {
                    const int r = (u + RO / 2) % RO;
                    const int row = j + r * (L / RO);
                    // V_j = sigma(z_j) dz F[|A_j|^2 A_j] exp(-i beta(w, z_j) - int G)   (Eq. (6))
                    const C v = cscale(cmul(vout[q][r], cconj(expi_turns_poly(pr.next()))), (float)nc.post);
                    if (MPA_DBG_OK(p.dbg, dst + (long long)row * rs, sizeof(C))) dst[(long long)row * rs] = v;
                }
            }
        }
    }
    // this thread's copies must land before the block's shared memory is released
    cp_async_wait_all();
}

}  // namespace mpa
