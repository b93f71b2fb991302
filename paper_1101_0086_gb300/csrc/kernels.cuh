// Kernels of the MPA node transform (MPA steps 2-5) and of the split-step
// comparator, on the four-step factorisation N = N1 * N2.
//
// A spectrum in natural order, k = k1 + N1 k2, is viewed as an N2 x N1
// row-major matrix.  The inverse transform is a column pass (length-N2 DFTs
// over k2, then the factor W_N^{-n2 k1}) followed by a row pass (length-N1
// DFTs over k1); row n2 then holds A(t) at t-index N2 n1 + n2 for
// n1 = 0..N1-1.  Because |A|^2 A (MPA step 4) and the split-step rotation
// are pointwise, the row pass forms them right there and starts the forward
// transform (length-N1 DFTs over n1, factor W_N^{+n2 k1}) without any
// transpose; the next column pass finishes it (length-N2 DFTs over n2) and
// leaves the spectrum in natural order again.
//
//   KC (column pass)  modes: MPA_PRE  phase exp(i beta_j) * exp(int G) -> inverse
//                             MPA_POST forward -> exp(-i beta_j) * sigma dz / exp(int G)  (V_j of Eq. (6))
//                             SS_STEP  forward -> linear step of Eq. (4) -> inverse
//                             FWD      forward only        INV  inverse only
//   KR (row pass)     modes: MPA  inverse -> 1/N -> |A|^2 A -> forward
//                             SS   inverse -> 1/N -> A exp(i s |A|^2) -> forward
//                             FWD  forward only        INV  inverse -> 1/N
//   SCAN              Eq. (6) trapezoid partial sums over the nodes for
//                     every frequency, fused with step 7 on the last iteration.
#pragma once

#include <type_traits>

#include "device.cuh"

namespace mpa {

enum { KC_MPA_PRE = 0, KC_MPA_POST = 1, KC_SS_STEP = 2, KC_FWD = 3, KC_INV = 4 };
// KR_MPA_KEEP: KR_MPA that also writes A(t) to keep (the reverse mode's
// forward recompute keeps it for the adjoint of the Kerr term)
enum { KR_MPA = 0, KR_SS = 1, KR_FWD = 2, KR_INV = 3, KR_MPA_KEEP = 4 };

// Debug build (MPA_DEBUG_BOUNDS=1): the global accesses of the MPA passes,
// the scan and the on-chip node transform are checked against the range of
// the launch's buffers (a plan's or batch's workspace, [lo, hi)); an access
// outside it sets ERR_BOUNDS in the error word and is skipped (a load reads
// zero), so a bad index is reported instead of touching memory it should
// not.  lo == nullptr (launches on caller buffers) checks nothing.  Release
// builds compile every check to true.
#ifndef MPA_DEBUG_BOUNDS
#define MPA_DEBUG_BOUNDS 0
#endif
enum { ERR_BOUNDS = 8u };
struct DbgRange {
    const char* lo;
    const char* hi;
    unsigned int* err;
};
__device__ __forceinline__ bool dbg_in(const DbgRange& d, const void* a, size_t bytes) {
    if (!d.lo) return true;
    const char* c = static_cast<const char*>(a);
    if (c >= d.lo && c + bytes <= d.hi) return true;
    atomicOr(d.err, (unsigned)ERR_BOUNDS);
    return false;
}
#if MPA_DEBUG_BOUNDS
#define MPA_DBG_OK(d, ptr, bytes) ::mpa::dbg_in((d), (ptr), (bytes))
#else
#define MPA_DBG_OK(d, ptr, bytes) true
#endif

// A launch covers nl links x npl nodes each (node index within the launch
// n = l npl + jn); a single link is nl = 1.
template <typename T> struct KCParams {
    const cx<T>* src;
    long long src_stride;   // elements between consecutive nodes of a link's source (0: shared source)
    long long src_lstride;  // elements between links' sources
    cx<T>* dst;
    long long dst_stride;
    long long dst_lstride;
    const cx<T>* src0;      // if non-null: the source of node jn == 0 of link l is src0 + l src0_lstride
    long long src0_lstride;
    long long N;
    int logN;
    int N1, logN1;
    long long ncols;        // nl * npl * N1 columns in this launch
    int npl;                // nodes per link in this launch
    const NodeC* nodes;     // MPA: constants of link l, node jn at nodes[loff[l] + jn]
    const int* loff;
    NodeC flow;             // SS: constants of the linear step
    unsigned int* err;      // error word of the staged column pass (null: kc_kernel only)
    long long spin_limit;   // polls of each bounded wait of the staged column pass
    // staged column pass only: sources other than src0 (tiled_in) / the
    // destination (tiled_out) hold node spectra in the tile layout (column
    // block b = k1 / G of a node as G x N2 contiguous elements, element
    // (k2, k1 mod G) at b G N2 + k2 G + k1 mod G) instead of natural order
    int tiled_in, tiled_out;
    DbgRange dbg;  // checked range of the debug build
};

template <typename T> struct KRParams {
    cx<T>* data;  // nrows contiguous rows of length N1
    long long nrows;
    long long N;
    int logN;
    int N2;
    T inv_n;  // 1/N
    T rot;    // SS: int sigma over the step
    cx<T>* keep;  // KR_MPA_KEEP: receives A(t), rows laid out as data
    unsigned int* err;       // error word of the staged row pass (null: kr_kernel only)
    long long spin_limit;    // polls of each bounded wait of the staged row pass
    DbgRange dbg;            // checked range of the debug build
};

// Column pass geometry for column length L: G columns per tile, NT threads.
template <typename T, int L> struct KCGeom {
    typedef Tiling<T> P;
    static constexpr int G = (P::TE / L) > P::CMIN ? (P::TE / L) : P::CMIN;
    static constexpr int TE = G * L;
    static constexpr int NT = TE / P::E;
    static constexpr int OSH = 5;  // outer-factor two-level split of n2
    static constexpr int OLO = L < 32 ? L : 32;
    static constexpr int OHI = L > 32 ? L / 32 : 1;
    static constexpr size_t smem_elems = (size_t)TE + (TE >> P::PSH) + 1 + TwDims<L>::NLO + TwDims<L>::NHI +
                                         (size_t)G * (OLO + OHI);
    // FP32: + the exp(2 pi i m/1024) table of the per-element phases
    static constexpr size_t smem_bytes = smem_elems * sizeof(cx<T>);
};

template <typename T, int L> struct KRGeom {
    typedef Tiling<T, 1> P;
    static constexpr int G = (P::TE / L) > 1 ? (P::TE / L) : 1;
    static constexpr int TE = G * L;
    static constexpr int NT = TE / P::E;
    static constexpr int OSH = 7;  // outer-factor split of k1
    static constexpr int OLO = L < 128 ? L : 128;
    static constexpr int OHI = L > 128 ? L / 128 : 1;
    static constexpr size_t smem_elems = (size_t)TE + (TE >> P::PSH) + 1 + TwDims<L>::NLO + TwDims<L>::NHI +
                                         (size_t)G * (OLO + OHI);
    static constexpr size_t smem_bytes = smem_elems * sizeof(cx<T>);
};

__device__ __forceinline__ long long signed_k(long long k, long long N) { return k < (N >> 1) ? k : k - N; }

// Global load of data another CTA of the same (persistent) kernel may have
// written: CG = true reads through L2 only (L1 is not coherent within a
// kernel); separate launches use ordinary loads.
template <bool CG, class V> __device__ __forceinline__ V ldx(const V* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Kahan-compensated s += v (c carries the lost low-order part).
template <typename T> __device__ __forceinline__ void kahan_add(T& s, T& c, T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// L2 prefetch distance of the FP32 column and row passes, in tiles: each CTA
// asks L2 for the tile that the CTA this many launches later will load (0:
// off).  One wave (2 CTAs x 152 SMs) ahead speeds the row pass up by 9 %
// (its tiles are contiguous); the column pass's strided 64-byte rows are
// slower with it.
#ifndef MPA_L2PF_KC
#define MPA_L2PF_KC 0
#endif
// the forward column pass (V_j, MPA_POST) reads what the row pass just
// wrote; one wave ahead it gains 3.7 % (3815 -> 3957 GB/s on the 2^20 link,
// split 2^12 x 2^8) while the inverse pass loses 6.6 % with it
#ifndef MPA_L2PF_KC_POST
#define MPA_L2PF_KC_POST 304
#endif
#ifndef MPA_L2PF_KR
#define MPA_L2PF_KR 304
#endif

__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

#ifndef MPA_KC_MINB
#define MPA_KC_MINB 2
#endif
#ifndef MPA_KR_MINB
#define MPA_KR_MINB 2
#endif
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(KCGeom<T, L>::NT, KCGeom<T, L>::NT <= 256 ? MPA_KC_MINB : 1)
    kc_kernel(const KCParams<T> p) {
    typedef cx<T> C;
    typedef KCGeom<T, L> Gm;
    typedef Tiling<T> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    constexpr bool FWD = (MODE == KC_MPA_POST || MODE == KC_SS_STEP || MODE == KC_FWD);
    constexpr bool INV = (MODE == KC_MPA_PRE || MODE == KC_SS_STEP || MODE == KC_INV);
    // forward: small radix first, so it ends with an RMAX pass that meets the
    // inverse's first RMAX pass in registers (split-step column pass)
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_COL, P::PSH, true> XF;
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_COL, P::PSH, false> XI;
    static_assert(!(FWD && INV) || XF::RL == XI::R0, "forward/inverse junction radix");
    typedef typename std::conditional<FWD, XF, XI>::type XA;  // first transform
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;  // [OLO][G]
    C* ohi = olo + G * Gm::OLO;     // [OHI][G]
    const int tid = threadIdx.x;
    const long long col0 = (long long)blockIdx.x * G;
    const int N1m = p.N1 - 1;
    constexpr bool FAST = sizeof(T) == 4;  // FP32: finite-difference phases + polynomial exp

    tw_init<T, L>(thi, tlo, tid, NT);
    if constexpr (INV) {
        // W_N^{-n2 k1} for the tile's columns: olo[m][g] = W^{-k1 m}, ohi[h][g] = W^{-k1 32 h}
        for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
            const int g = i % G, m = i / G;
            const long long k1 = (col0 + g) & N1m;
            if (m < Gm::OLO) olo[m * G + g] = expi_ratio<T>(-k1 * m, p.logN);
            else ohi[(m - Gm::OLO) * G + g] = expi_ratio<T>(-k1 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
        }
    }
    __syncthreads();

    // ---- load: element j + r L/R0 of column col0 + g, straight into registers
    C vin[XA::Q0][XA::R0];
#pragma unroll
    for (int q = 0; q < XA::Q0; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, XA::R0>(tid + q * NT, j, g);
        const long long col = col0 + g;
        const bool ok = col < p.ncols;
        const int node = ok ? (int)(col >> p.logN1) : 0;
        const int l = node / p.npl, jn = node - l * p.npl;
        const long long c = col & N1m;
        const C* src = (p.src0 && jn == 0) ? p.src0 + l * p.src0_lstride + c
                                           : p.src + l * p.src_lstride + jn * p.src_stride + c;
        NodeC nc{};
        if constexpr (MODE == KC_MPA_PRE) {
            if (MPA_DBG_OK(p.dbg, p.loff + l, sizeof(int)) && MPA_DBG_OK(p.dbg, p.nodes + p.loff[l] + jn, sizeof(NodeC)))
                nc = p.nodes[p.loff[l] + jn];
        }
        unsigned long long th[XA::R0];
        if constexpr (FAST && MODE == KC_MPA_PRE)
            phase_run<XA::R0>(c + (long long)j * p.N1, (long long)p.N1 * (L / XA::R0), nc, th);
#pragma unroll
        for (int r = 0; r < XA::R0; ++r) {
            const int row = j + r * (L / XA::R0);
            C v = ok && MPA_DBG_OK(p.dbg, src + (long long)row * p.N1, sizeof(C)) ? src[(long long)row * p.N1]
                                                                                  : mkc(T(0), T(0));
            if constexpr (MODE == KC_MPA_PRE) {
                // MPA step 2: A_hat_j = psi_j exp(i beta(w, z_j) + int G)
                C ph;
                if constexpr (FAST) ph = expi_turns_poly(th[r]);
                else ph = expi_turns<T>(phase_q64(signed_k(c + (long long)row * p.N1, p.N), nc));
                v = cscale(cmul(v, ph), (T)nc.pre);
            }
            vin[q][r] = v;
        }
    }

    constexpr int L2PF = MODE == KC_MPA_POST ? MPA_L2PF_KC_POST : MPA_L2PF_KC;
    if constexpr (FAST && L2PF > 0) {
        const long long tb = (long long)blockIdx.x + L2PF;
        if (tb < (long long)gridDim.x) {
            // the first node's columns of that tile (all of it when G <= N1)
            const long long col = tb * G;
            const int node = (int)(col >> p.logN1);
            const int l = node / p.npl, jn = node - l * p.npl;
            const long long c = col & N1m;
            const C* src = (p.src0 && jn == 0) ? p.src0 + l * p.src0_lstride + c
                                               : p.src + l * p.src_lstride + jn * p.src_stride + c;
            long long w = p.ncols - col < G ? p.ncols - col : G;
            if (w > p.N1 - c) w = p.N1 - c;
            // whole 128-byte L2 lines: a tile narrower than a line prefetches
            // the line once (the tile at its start), the others skip
            constexpr long long LINE = 128 / (long long)sizeof(C);
            bool go = true;
            if (w < LINE) {
                go = (c % LINE) == 0 && c + LINE <= p.N1;
                w = LINE;
            }
            if (go)
                for (int r = tid; r < L; r += NT) prefetch_l2(src + (long long)r * p.N1, (unsigned)(w * sizeof(C)));
        }
    }

    // ---- transforms
    constexpr int QO = INV ? XI::QL : XF::QL, RO = INV ? XI::RL : XF::RL;
    C vout[QO][RO];
    if constexpr (FWD && INV) {
        C vm[XF::QL][XF::RL];
        XF::run(vin, vm, s, thi, tlo);
        // exact linear step exp(i beta(w; za, zb) + int G) between the kicks of Eq. (4)
#pragma unroll
        for (int q = 0; q < XF::QL; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, G, XF::RL>(tid + q * NT, j, g);
            const long long c = (col0 + g) & N1m;
            unsigned long long th[XF::RL];
            if constexpr (FAST) phase_run<XF::RL>(c + (long long)j * p.N1, (long long)p.N1 * (L / XF::RL), p.flow, th);
#pragma unroll
            for (int r = 0; r < XF::RL; ++r) {
                const int row = j + r * (L / XF::RL);
                C ph;
                if constexpr (FAST) ph = expi_turns_poly(th[r]);
                else ph = expi_turns<T>(phase_q64(signed_k(c + (long long)row * p.N1, p.N), p.flow));
                vm[q][r] = cscale(cmul(vm[q][r], ph), (T)p.flow.pre);
            }
        }
        XI::run(vm, vout, s, thi, tlo);
    } else if constexpr (FWD) {
        XF::run(vin, vout, s, thi, tlo);
    } else {
        XI::run(vin, vout, s, thi, tlo);
    }

    // ---- epilogue and store: element j + r L/RO of column col0 + g
#pragma unroll
    for (int q = 0; q < QO; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, RO>(tid + q * NT, j, g);
        const long long col = col0 + g;
        if (col >= p.ncols) continue;
        const int node = (int)(col >> p.logN1);
        const int l = node / p.npl, jn = node - l * p.npl;
        const long long c = col & N1m;
        C* dst = p.dst + l * p.dst_lstride + jn * p.dst_stride + c;
        NodeC nc{};
        if constexpr (MODE == KC_MPA_POST) {
            if (MPA_DBG_OK(p.dbg, p.loff + l, sizeof(int)) && MPA_DBG_OK(p.dbg, p.nodes + p.loff[l] + jn, sizeof(NodeC)))
                nc = p.nodes[p.loff[l] + jn];
        }
        unsigned long long th[RO];
        if constexpr (FAST && MODE == KC_MPA_POST)
            phase_run<RO>(c + (long long)j * p.N1, (long long)p.N1 * (L / RO), nc, th);
        // rows j + r L/RO share their low outer-factor index when L/RO is a
        // multiple of the low table's length: one lookup per butterfly
        constexpr bool HOIST = (L / RO) % Gm::OLO == 0;
        C wlo = mkc(T(1), T(0));
        if constexpr (INV && HOIST) wlo = olo[(j & (Gm::OLO - 1)) * G + g];
#pragma unroll
        for (int r = 0; r < RO; ++r) {
            const int row = j + r * (L / RO);
            C v = vout[q][r];
            if constexpr (INV) {
                // four-step factor W_N^{-n2 k1}, n2 = row
                C w = HOIST ? wlo : olo[(row & (Gm::OLO - 1)) * G + g];
                if constexpr (Gm::OHI > 1) w = cmul(ohi[(row >> Gm::OSH) * G + g], w);
                v = cmul(v, w);
            }
            if constexpr (MODE == KC_MPA_POST) {
                // V_j = sigma(z_j) dz F[|A_j|^2 A_j] exp(-i beta(w, z_j) - int G)   (Eq. (6))
                C ph;
                if constexpr (FAST) ph = expi_turns_poly(th[r]);
                else ph = expi_turns<T>(phase_q64(signed_k(c + (long long)row * p.N1, p.N), nc));
                v = cscale(cmul(v, cconj(ph)), (T)nc.post);
            }
            if (MPA_DBG_OK(p.dbg, dst + (long long)row * p.N1, sizeof(C))) dst[(long long)row * p.N1] = v;
        }
    }
}

template <typename T, int L, int MODE>
__global__ void __launch_bounds__(KRGeom<T, L>::NT, KRGeom<T, L>::NT <= 256 ? MPA_KR_MINB : 1)
    kr_kernel(const KRParams<T> p) {
    typedef cx<T> C;
    typedef KRGeom<T, L> Gm;
    typedef Tiling<T, 1> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    constexpr bool INV = (MODE != KR_FWD);
    constexpr bool FWD = (MODE != KR_INV);
    // inverse: small radix last, forward: small radix first, so the two meet
    // in registers around the pointwise step
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_ROW, P::PSH, false> XI;
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_ROW, P::PSH, true> XF;
    static_assert(!(FWD && INV) || XI::RL == XF::R0, "inverse/forward junction radix");
    typedef typename std::conditional<INV, XI, XF>::type XA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;  // [G][OLO]
    C* ohi = olo + G * Gm::OLO;     // [G][OHI]
    const int tid = threadIdx.x;
    const long long row0 = (long long)blockIdx.x * G;

    tw_init<T, L>(thi, tlo, tid, NT);
    if constexpr (FWD) {
        // W_N^{+n2 k1} for the tile's rows: olo[g][m] = W^{n2 m}, ohi[g][h] = W^{n2 128 h}
        for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
            const int g = i / (Gm::OLO + Gm::OHI), m = i % (Gm::OLO + Gm::OHI);
            const long long n2 = (row0 + g) & (p.N2 - 1);
            if (m < Gm::OLO) olo[g * Gm::OLO + m] = expi_ratio<T>(n2 * m, p.logN);
            else ohi[g * Gm::OHI + (m - Gm::OLO)] = expi_ratio<T>(n2 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
        }
    }
    __syncthreads();

    C vin[XA::Q0][XA::R0];
#pragma unroll
    for (int q = 0; q < XA::Q0; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XA::R0>(tid + q * NT, j, g);
        const bool ok = row0 + g < p.nrows;
        const C* src = p.data + (row0 + g) * L;
#pragma unroll
        for (int r = 0; r < XA::R0; ++r)
            vin[q][r] = ok && MPA_DBG_OK(p.dbg, src + j + r * (L / XA::R0), sizeof(C)) ? src[j + r * (L / XA::R0)]
                                                                                     : mkc(T(0), T(0));
    }

    if constexpr (sizeof(T) == 4 && MPA_L2PF_KR > 0) {
        const long long tb = (long long)blockIdx.x + MPA_L2PF_KR;
        const long long r0 = tb * G;
        if (tb < (long long)gridDim.x && r0 < p.nrows) {
            const long long nr = p.nrows - r0 < G ? p.nrows - r0 : G;
            const long long bytes = nr * L * (long long)sizeof(C);  // contiguous rows
            const C* base = p.data + r0 * L;
            for (long long o = (long long)tid * 256; o < bytes; o += (long long)NT * 256)
                prefetch_l2(reinterpret_cast<const char*>(base) + o, (unsigned)(bytes - o < 256 ? bytes - o : 256));
        }
    }

    constexpr int QO = FWD ? XF::QL : XI::QL, RO = FWD ? XF::RL : XI::RL;
    C vout[QO][RO];
    if constexpr (INV && FWD) {
        C vm[XI::QL][XI::RL];
        XI::run(vin, vm, s, thi, tlo);
#pragma unroll
        for (int q = 0; q < XI::QL; ++q) {
            C* kp = nullptr;
            int jk = 0;
            if constexpr (MODE == KR_MPA_KEEP) {
                int g;
                bmap<LAYOUT_ROW, L, G, XI::RL>(tid + q * NT, jk, g);
                if (row0 + g < p.nrows) kp = p.keep + (row0 + g) * L;
            }
#pragma unroll
            for (int r = 0; r < XI::RL; ++r) {
                C a = cscale(vm[q][r], p.inv_n);  // A(t) (MPA step 3 / SS inverse)
                if constexpr (MODE == KR_MPA_KEEP) {
                    if (kp && MPA_DBG_OK(p.dbg, kp + jk + r * (L / XI::RL), sizeof(C))) kp[jk + r * (L / XI::RL)] = a;
                }
                const T pw = a.x * a.x + a.y * a.y;
                if constexpr (MODE == KR_MPA || MODE == KR_MPA_KEEP) {
                    a = cscale(a, pw);  // |A|^2 A (MPA step 4)
                } else {
                    T sn, cs;  // A exp(i s |A|^2), the nonlinear step of Eq. (4)
                    sincos_kerr(p.rot * pw, &sn, &cs);
                    a = cmul(a, mkc(cs, sn));
                }
                vm[q][r] = a;
            }
        }
        XF::run(vm, vout, s, thi, tlo);
    } else if constexpr (INV) {
        XI::run(vin, vout, s, thi, tlo);
    } else {
        XF::run(vin, vout, s, thi, tlo);
    }

#pragma unroll
    for (int q = 0; q < QO; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, RO>(tid + q * NT, j, g);
        if (row0 + g >= p.nrows) continue;
        C* dst = p.data + (row0 + g) * L;
        constexpr bool HOIST = (L / RO) % Gm::OLO == 0;  // one low-table lookup per butterfly
        C wlo = mkc(T(1), T(0));
        if constexpr (FWD && HOIST) wlo = olo[g * Gm::OLO + (j & (Gm::OLO - 1))];
#pragma unroll
        for (int r = 0; r < RO; ++r) {
            const int l = j + r * (L / RO);  // k1
            C v = vout[q][r];
            if constexpr (FWD) {
                C w = HOIST ? wlo : olo[g * Gm::OLO + (l & (Gm::OLO - 1))];
                if constexpr (Gm::OHI > 1) w = cmul(ohi[g * Gm::OHI + (l >> Gm::OSH)], w);
                v = cmul(v, w);
            } else {
                v = cscale(v, p.inv_n);
            }
            if (MPA_DBG_OK(p.dbg, dst + l, sizeof(C))) dst[l] = v;
        }
    }
}

// ------------------------------------------------------------------
// Whole node transform on chip (MPA steps 2-4 and the weight of Eq. (6)) for
// N small enough that one spectrum fits in a CTA's shared memory (N <= 2^14
// FP32, 2^13 FP64): G = TE/N nodes per CTA, each a row of the row-pass tile
// layout holding its spectrum in natural order:
//   A_hat = psi_j exp(i beta_j + int G)        (phase at the load, step 2)
//   A = F^-1[A_hat]; U = |A|^2 A; F[U]          (steps 3-4, in shared memory)
//   V_j = F[U] sigma_j dz exp(-i beta_j - int G)   (at the store, Eq. (6))
// One HBM (or L2) round trip per node instead of the three of the column,
// row and column passes, no four-step outer factors.  Node addressing as in
// KCParams (nl links x npl nodes, psi_0 shared by node 0).
template <typename T> struct KNParams {
    const cx<T>* src;
    long long src_stride, src_lstride;
    const cx<T>* src0;  // if non-null: the source of node jn == 0 of link l is src0 + l src0_lstride
    long long src0_lstride;
    cx<T>* dst;
    long long dst_stride, dst_lstride;
    long long nrows;    // nl * npl nodes in this launch
    int npl;
    const NodeC* nodes;  // link l, node jn at nodes[loff[l] + jn]
    const int* loff;
    T inv_n;
    DbgRange dbg;  // checked range of the debug build
};

template <typename T, int L> struct KNGeom {
    typedef KRGeom<T, L> R;
    static constexpr int G = R::G, TE = R::TE, NT = R::NT;
    typedef Tiling<T, 1> P;
    static constexpr size_t smem_bytes =
        ((size_t)TE + (TE >> P::PSH) + 1 + TwDims<L>::NLO + TwDims<L>::NHI) * sizeof(cx<T>);
};

// The node rows row0 .. row0 + G - 1 of a launch (one tile) through steps
// 2-4 and the weight of Eq. (6); the block's threads and shared memory.
template <typename T, int L, bool CG>
__device__ __forceinline__ void kn_tile(const KNParams<T>& p, long long row0, unsigned char* smem_raw) {
    typedef cx<T> C;
    typedef KNGeom<T, L> Gm;
    typedef Tiling<T, 1> P;
    constexpr int G = Gm::G, NT = Gm::NT, TE = Gm::TE;
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_ROW, P::PSH, false> XI;
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_ROW, P::PSH, true> XF;
    static_assert(XI::RL == XF::R0, "inverse/forward junction radix");
    constexpr bool FAST = sizeof(T) == 4;  // FP32: finite-difference phases + polynomial exp
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    const int tid = threadIdx.x;

    tw_init<T, L>(thi, tlo, tid, NT);
    __syncthreads();

    // ---- load node spectra (natural order, k = element index) and step 2
    C vin[XI::Q0][XI::R0];
#pragma unroll
    for (int q = 0; q < XI::Q0; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XI::R0>(tid + q * NT, j, g);
        const long long row = row0 + g;
        const bool ok = row < p.nrows;
        const int node = ok ? (int)row : 0;
        const int l = node / p.npl, jn = node - l * p.npl;
        const C* src = (p.src0 && jn == 0) ? p.src0 + l * p.src0_lstride : p.src + l * p.src_lstride + jn * p.src_stride;
        NodeC nc{};
        if (MPA_DBG_OK(p.dbg, p.loff + l, sizeof(int)) && MPA_DBG_OK(p.dbg, p.nodes + p.loff[l] + jn, sizeof(NodeC)))
            nc = p.nodes[p.loff[l] + jn];
        unsigned long long th[XI::R0];
        if constexpr (FAST) phase_run<XI::R0>(j, L / XI::R0, nc, th);
#pragma unroll
        for (int r = 0; r < XI::R0; ++r) {
            const int k = j + r * (L / XI::R0);
            C v = ok && MPA_DBG_OK(p.dbg, src + k, sizeof(C)) ? ldx<CG>(src + k) : mkc(T(0), T(0));
            C ph;
            if constexpr (FAST) ph = expi_turns_poly(th[r]);
            else ph = expi_turns<T>(phase_q64(signed_k(k, L), nc));
            vin[q][r] = cscale(cmul(v, ph), (T)nc.pre);
        }
    }

    // ---- steps 3-4: inverse transform, 1/N, |A|^2 A, forward transform
    C vm[XI::QL][XI::RL];
    XI::run(vin, vm, s, thi, tlo);
#pragma unroll
    for (int q = 0; q < XI::QL; ++q) {
#pragma unroll
        for (int r = 0; r < XI::RL; ++r) {
            const C a = cscale(vm[q][r], p.inv_n);
            vm[q][r] = cscale(a, a.x * a.x + a.y * a.y);
        }
    }
    C vout[XF::QL][XF::RL];
    XF::run(vm, vout, s, thi, tlo);

    // ---- V_j (Eq. (6)) and the store, natural order
#pragma unroll
    for (int q = 0; q < XF::QL; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XF::RL>(tid + q * NT, j, g);
        const long long row = row0 + g;
        if (row >= p.nrows) continue;
        const int node = (int)row;
        const int l = node / p.npl, jn = node - l * p.npl;
        C* dst = p.dst + l * p.dst_lstride + jn * p.dst_stride;
        NodeC nc{};
        if (MPA_DBG_OK(p.dbg, p.loff + l, sizeof(int)) && MPA_DBG_OK(p.dbg, p.nodes + p.loff[l] + jn, sizeof(NodeC)))
            nc = p.nodes[p.loff[l] + jn];
        unsigned long long th[XF::RL];
        if constexpr (FAST) phase_run<XF::RL>(j, L / XF::RL, nc, th);
#pragma unroll
        for (int r = 0; r < XF::RL; ++r) {
            const int k = j + r * (L / XF::RL);
            C ph;
            if constexpr (FAST) ph = expi_turns_poly(th[r]);
            else ph = expi_turns<T>(phase_q64(signed_k(k, L), nc));
            if (MPA_DBG_OK(p.dbg, dst + k, sizeof(C))) dst[k] = cscale(cmul(vout[q][r], cconj(ph)), (T)nc.post);
        }
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(KNGeom<T, L>::NT, KNGeom<T, L>::NT <= 256 ? MPA_KR_MINB : 1)
    kn_kernel(const KNParams<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    kn_tile<T, L, false>(p, (long long)blockIdx.x * KNGeom<T, L>::G, smem_raw);
}

// ------------------------------------------------------------------
// Wavefront column pass (FP32): one CTA owns one column tile of one block
// of B consecutive nodes at one Picard level and walks the nodes in order:
//   forward column DFTs (finishing F[|A_j|^2 A_j])
//   V_j = F[...] exp(-i beta_j) sigma_j dz / exp(int G)          (Eq. (6))
//   psi^{(n+1)}_j = psi_0 + i (R + V_j/2),  R += V_j              (step 5)
//   A_hat = psi^{(n+1)}_j exp(i beta_j + int G) and the inverse column DFTs
//   of level n+1 (steps 2-3), written back over the node's buffer.
// R (the trapezoid running sum of this level, Kahan-compensated, the
// compensation kept in shared memory) persists across the block in
// registers and across blocks in global memory.  The phase of node j is
// evaluated once for both directions.  On the last level the inverse
// transform is instead that of the next block's first iteration for the
// node S B further on (psi_0 exp(i beta + int G)), and the node-M value
// psi_0 + i (R + V_M/2) is emitted in FP64 for step 7.
struct KCWJob {
    int level, slot, node_first, n_nodes, head_first, n_head, last;
};

struct KCWParams {
    float2* work;           // slots of B node buffers
    long long slot_stride;  // elements between slots
    long long N;
    int logN, N1, logN1, M;
    const NodeC* nodes;     // this interval's constants, node j at nodes[j]
    const float2* psi0;     // psi_0 (complex64, natural order)
    const float2* v0;       // V_0 (complex64) for blocks that start at node 1
    float2* Rg;             // [levels][N] running sums
    float2* Cg;             // [levels][N] Kahan compensations
    double2* D;             // R + V_M/2 at node M (so psi_M = psi_0 + i D), FP64
    int n_jobs;
    KCWJob job[8];  // one per Picard level (n_iter <= 8)
};

// Tile of the wavefront column pass: MPA_KCW_TE elements (at least 4
// columns); the running sums and compensations take 16 bytes per element of
// shared memory, so 4096-element tiles (about 102 KB with the transform
// tile) let two CTAs share an SM and 8192-element ones (about 200 KB) one.
#ifndef MPA_KCW_TE
#define MPA_KCW_TE 4096
#endif
#ifndef MPA_KCW_MINB
#define MPA_KCW_MINB 2
#endif
template <int L> struct KCWGeom {
    typedef Tiling<float, 2> P;
    static constexpr int G = (MPA_KCW_TE / L) > 4 ? (MPA_KCW_TE / L) : 4, TE = G * L, NT = TE / P::E;
    static constexpr int OSH = 5, OLO = L < 32 ? L : 32, OHI = L > 32 ? L / 32 : 1;
    // float2 offset of the running sums (float4 per element): rounded up to
    // an even count so the array starts on a 16-byte boundary
    static constexpr size_t RC_OFF =
        (((size_t)TE + (TE >> P::PSH) + 1 + TwDims<L>::NLO + TwDims<L>::NHI + (size_t)G * (OLO + OHI)) + 1) & ~(size_t)1;
    static constexpr size_t smem_bytes = RC_OFF * sizeof(float2) + (size_t)TE * sizeof(float4);
};

// The node loop of one job; LAST selects the last Picard level (heads of
// the next blocks instead of the next level, and the node-M output).
template <int L, bool LAST>
__device__ __forceinline__ void kcw_job(const KCWParams& p, const KCWJob& job, float2* s, const float2* thi,
                                        const float2* tlo, const float2* olo, const float2* ohi, float4* rc,
                                        int col0) {
    typedef float2 C;
    typedef KCWGeom<L> Gm;
    typedef Tiling<float, 2> P;
    constexpr int G = Gm::G, NT = Gm::NT;
    typedef Xform<float, L, G, NT, P::RMAX, +1, LAYOUT_COL, P::PSH, true> XF;
    typedef Xform<float, L, G, NT, P::RMAX, -1, LAYOUT_COL, P::PSH, false> XI;
    constexpr int QJ = XF::QL, RJ = XF::RL;
    const int tid = threadIdx.x;
    const long long N = p.N;
    const long long D = (long long)p.N1 * (L / RJ);

    // running sums of this level (and Kahan compensations) for the thread's
    // junction elements, kept in shared memory across the node loop
#pragma unroll
    for (int q = 0; q < QJ; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, RJ>(tid + q * NT, j, g);
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
            const long long k = (col0 + g) + (long long)(j + r * (L / RJ)) * p.N1;
            float4 e;
            if (job.node_first == 1) {
                const float2 v = p.v0[k];
                e = make_float4(0.5f * v.x, 0.5f * v.y, 0.f, 0.f);  // V_0 / 2
            } else {
                const float2 rv = p.Rg[(long long)job.level * N + k], cv = p.Cg[(long long)job.level * N + k];
                e = make_float4(rv.x, rv.y, cv.x, cv.y);
            }
            rc[(q * RJ + r) * NT + tid] = e;
        }
    }

    float2* slot = p.work + (long long)job.slot * p.slot_stride;
    for (int i = 0; i < job.n_nodes; ++i) {
        const int jn = job.node_first + i;
        float2* buf = slot + (long long)i * N;
        // ---- forward column DFTs of node jn (first pass straight from global)
        C vin[XF::Q0][XF::R0];
#pragma unroll
        for (int q = 0; q < XF::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, G, XF::R0>(tid + q * NT, j, g);
            const C* src = buf + col0 + g;
#pragma unroll
            for (int r = 0; r < XF::R0; ++r) vin[q][r] = src[(long long)(j + r * (L / XF::R0)) * p.N1];
        }
        C v[QJ][RJ];
        XF::run(vin, v, s, thi, tlo);
        const bool head = LAST && i < job.n_head;
        const NodeC nc = p.nodes[jn];
        const float post = (float)nc.post;
#pragma unroll
        for (int q = 0; q < QJ; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, G, RJ>(tid + q * NT, j, g);
            const long long c = col0 + g;
            // elements in s order: s = -RJ/2 .. RJ/2-1, r = (s + RJ) mod RJ, k' = c + N1 (j + s L/RJ)
            const long long kf = c + (long long)p.N1 * j - (long long)(RJ / 2) * D;
            PhaseRun pr(kf, D, nc);
            if constexpr (!LAST) {
                const float pre = (float)nc.pre;
#pragma unroll
                for (int t = 0; t < RJ; ++t) {
                    const int r = (t + RJ / 2) % RJ;
                    const long long k = c + (long long)(j + r * (L / RJ)) * p.N1;
                    const C ph = expi_turns_poly(pr.next());
                    // V_j (Eq. (6)) and psi^{(n+1)}_j = psi_0 + i (R + V_j/2) (step 5)
                    const C V = cscale(cmul(v[q][r], cconj(ph)), post);
                    float4 e = rc[(q * RJ + r) * NT + tid];  // (R, compensation)
                    const float2 p0 = p.psi0[k];
                    const float sx = (e.x - e.z) + 0.5f * V.x, sy = (e.y - e.w) + 0.5f * V.y;
                    kahan_add(e.x, e.z, V.x);
                    kahan_add(e.y, e.w, V.y);
                    rc[(q * RJ + r) * NT + tid] = e;
                    // step 2 of the next iteration at the same node
                    v[q][r] = cscale(cmul(make_float2(p0.x - sy, p0.y + sx), ph), pre);
                }
            } else {
#pragma unroll
                for (int t = 0; t < RJ; ++t) {
                    const int r = (t + RJ / 2) % RJ;
                    const C ph = expi_turns_poly(pr.next());
                    const C V = cscale(cmul(v[q][r], cconj(ph)), post);
                    float4 e = rc[(q * RJ + r) * NT + tid];  // (R, compensation)
                    if (jn == p.M) {
                        // R + V_M/2 before adding V_M: psi_M = psi_0 + i D (FP64)
                        const long long k = c + (long long)(j + r * (L / RJ)) * p.N1;
                        p.D[k] = make_double2(((double)e.x - (double)e.z) + 0.5 * (double)V.x,
                                              ((double)e.y - (double)e.w) + 0.5 * (double)V.y);
                    }
                    kahan_add(e.x, e.z, V.x);
                    kahan_add(e.y, e.w, V.y);
                    rc[(q * RJ + r) * NT + tid] = e;
                }
                if (head) {
                    // first iteration of the node S B further on: psi_0 exp(i beta + int G)
                    const NodeC nh = p.nodes[job.head_first + i];
                    const float preh = (float)nh.pre;
                    PhaseRun ph2(kf, D, nh);
#pragma unroll
                    for (int t = 0; t < RJ; ++t) {
                        const int r = (t + RJ / 2) % RJ;
                        const long long k = c + (long long)(j + r * (L / RJ)) * p.N1;
                        v[q][r] = cscale(cmul(p.psi0[k], expi_turns_poly(ph2.next())), preh);
                    }
                }
            }
        }
        if (!LAST || head) {
            // ---- inverse column DFTs, four-step factor, store over the node buffer
            C vo[XI::QL][XI::RL];
            XI::run(v, vo, s, thi, tlo);
#pragma unroll
            for (int q = 0; q < XI::QL; ++q) {
                int j, g;
                bmap<LAYOUT_COL, L, G, XI::RL>(tid + q * NT, j, g);
                C* dst = buf + col0 + g;
#pragma unroll
                for (int r = 0; r < XI::RL; ++r) {
                    const int row = j + r * (L / XI::RL);
                    C w = olo[(row & (Gm::OLO - 1)) * G + g];
                    if constexpr (Gm::OHI > 1) w = cmul(ohi[(row >> Gm::OSH) * G + g], w);
                    dst[(long long)row * p.N1] = cmul(vo[q][r], w);
                }
            }
        }
    }

    // ---- running sums back to global memory for the next block
#pragma unroll
    for (int q = 0; q < QJ; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, RJ>(tid + q * NT, j, g);
#pragma unroll
        for (int r = 0; r < RJ; ++r) {
            const long long k = (col0 + g) + (long long)(j + r * (L / RJ)) * p.N1;
            const float4 e = rc[(q * RJ + r) * NT + tid];
            p.Rg[(long long)job.level * N + k] = make_float2(e.x, e.y);
            p.Cg[(long long)job.level * N + k] = make_float2(e.z, e.w);
        }
    }
}

template <int L>
__global__ void __launch_bounds__(KCWGeom<L>::NT, KCWGeom<L>::NT <= 256 ? MPA_KCW_MINB : 1)
    kcw_kernel(const KCWParams p) {
    typedef float2 C;
    typedef KCWGeom<L> Gm;
    typedef Tiling<float, 2> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;  // [OLO][G]
    C* ohi = olo + G * Gm::OLO;     // [OHI][G]
    float4* rc = reinterpret_cast<float4*>(s + Gm::RC_OFF);  // [E][NT] (R, compensation), 16-B aligned
    const int tid = threadIdx.x;
    const KCWJob job = p.job[blockIdx.y];
    const int col0 = blockIdx.x * G;  // column within a node (tiles never straddle nodes)

    tw_init<float, L>(thi, tlo, tid, NT);
    for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
        const int g = i % G, m = i / G;
        const long long k1 = col0 + g;
        if (m < Gm::OLO) olo[m * G + g] = expi_ratio<float>(-k1 * m, p.logN);
        else ohi[(m - Gm::OLO) * G + g] = expi_ratio<float>(-k1 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
    }
    __syncthreads();
    if (job.last) kcw_job<L, true>(p, job, s, thi, tlo, olo, ohi, rc, col0);
    else kcw_job<L, false>(p, job, s, thi, tlo, olo, ohi, rc, col0);
}

// Eq. (6) for every frequency k: running trapezoid sum over nodes j = 1..M
//   psi^{(n+1)}_l = psi_0 + i (V_0/2 + sum_{j=1}^{l-1} V_j + V_l/2),
// with V_j stored in psi[j] (node 0 holds V_0).  FP32 sums are Kahan-
// compensated; the final value at node M is formed in FP64.
//   mode 0: write psi^{(n+1)}_j into psi[j] (next iteration)
//   mode 1: step 7: state <- psi_M exp(i beta(w, z0+L) + int G) * gain, psi0c <- state
//   mode 2: out <- psi_M (FP64, no step 7)
//
// Run-time checks (text before the MPA steps: psi^{(n)} are Picard iterates
// that converge when L << z_nl).  Every level also measures its Picard
// increment at node M, Delta^{(n+1)} = psi^{(n+1)}_M - psi^{(n)}_M =
// i (D^{(n+1)} - D^{(n)}) with D the trapezoid sum of Eq. (6) at node M
// (D^{(0)} = 0), relative to |psi^{(n+1)}_M|:
//   rel_n = ||Delta^{(n+1)}|| / ||psi^{(n+1)}_M||   (sums over all frequencies).
// The last block of a link to finish (atomic ticket, no waiting) compares
// rel_n with rel_{n-1}: an increment that does not shrink, while above the
// rounding floor of the working precision, sets bit 1 of the error word
// (MPA_ERR_DIVERGED); a non-finite interval result sets bit 0.
// ERR_TIMEOUT (bit 2): a bounded wait of a persistent kernel ran out.
enum { ERR_NONFINITE = 1u, ERR_DIVERGED = 2u, ERR_TIMEOUT = 4u };
struct ConvState {
    double acc_d, acc_p;  // this level: sum |Delta|^2, sum |psi_M|^2
    double prev_rel;      // rel of the previous level of this interval
    double worst;         // largest rel_n / rel_{n-1} seen (contraction factor)
    unsigned int count;   // blocks of this level finished
    unsigned int pad;
};
// Device words of one group of links: the error word (bits above), one
// ConvState per link and D at node M per link (N complex64 each).
struct Monitor {
    unsigned int* err;
    ConvState* conv;
    float2* dprev;
    long long spin_limit;  // polls of each bounded wait of a persistent kernel
    DbgRange dbg;          // the debug build's checked range (the workspace)
};

// Natural index k = k1 + N1 k2 of position i of a node spectrum held in the
// tile layout of the staged column pass: column blocks of G = 2^logG columns,
// each G x N2 (N2 = 2^logL) contiguous, element (k2, k1 mod G) of block
// k1 / G at (k1 / G) G N2 + k2 G + k1 mod G.
__host__ __device__ __forceinline__ long long tile_to_natural(long long i, int logG, int logL, long long N) {
    const long long tb = i >> (logG + logL), rem = i & ((1ll << (logG + logL)) - 1);
    const long long k2 = rem >> logG, k1 = (tb << logG) + (rem & ((1ll << logG) - 1));
    return k1 + k2 * (N >> logL);
}

template <typename T> struct ScanParams {
    cx<T>* psi;          // link l's node j at psi + (l (M+1) + j) N
    long long N;
    int M;
    const cx<T>* psi0c;  // psi_0 in the working precision, link l at + l N
    double2* state;      // FP64 psi_0 in, A_hat(z0+L) out (mode 1), link l at + l N
    cx<T>* psi0c_out;    // mode 1: working-precision copy of the new state
    double2* out;        // mode 2
    int mode;
    const NodeC* nodes;  // node M of link l: nodes[loff[l] + M]
    const int* loff;
    const double* gain;  // amplifier gain at the interval end, per link
    unsigned int* err;
    // Picard increment check (skipped when conv is null): level n of n_iter
    ConvState* conv;     // per link
    float2* dprev;       // D^{(n)} at node M, link l at + l N (written unless last level)
    int level, n_iter;
    double floor_rel;    // increments below this relative size are rounding, not divergence
    // tile_logG > 0: psi and dprev hold node spectra in the tile layout of the
    // staged column pass (G = 2^tile_logG columns of N2 = 2^tile_logL rows,
    // N1 = N / N2 columns); psi0c, state and out stay in natural order
    int tile_logG, tile_logL;
    DbgRange dbg;  // checked range of the debug build
};

// Adds this block's sums to link l's accumulators; the last block of the
// level closes the level (comparison with the previous one, reset).
__device__ __forceinline__ void conv_close(ConvState* cs, unsigned int* err, double d2, double p2, int level,
                                           int last_level, double floor_rel, unsigned nblk) {
    __shared__ double red[2][32];  // one entry per warp (up to 1024 threads)
    __shared__ bool last_block;
    // warp sums, then the block's 8 warp sums by thread 0
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = d2;
        red[1][w] = p2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sd = 0.0, sp = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            sd += red[0][i];
            sp += red[1][i];
        }
        atomicAdd(&cs->acc_d, sd);
        atomicAdd(&cs->acc_p, sp);
        __threadfence();
        last_block = atomicAdd(&cs->count, 1u) == nblk - 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && last_block) {
        __threadfence();
        volatile ConvState* v = cs;
        const double sd = v->acc_d, sp = v->acc_p;
        const double rel = sp > 0.0 ? sqrt(sd / sp) : 0.0;
        if (level > 0) {
            const double q = v->prev_rel > 0.0 ? rel / v->prev_rel : (rel > 0.0 ? 1e300 : 0.0);
            if (q > v->worst) v->worst = q;
            if (!(rel < v->prev_rel) && rel > floor_rel) atomicOr(err, ERR_DIVERGED);
        }
        v->prev_rel = level == last_level ? 0.0 : rel;
        v->acc_d = 0.0;
        v->acc_p = 0.0;
        v->count = 0u;
    }
}

// Frequency k of link l (one thread each; a block of consecutive
// frequencies, nblk blocks per link).  N is a multiple of the block size (a
// power of two >= 256), so every thread has a frequency and takes part in
// the block reduction of the increment check.
// 8-byte global -> shared copy (cp.async.ca) and its commit / wait groups
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// S > 0 (FP32 only): the thread's V_j travel S nodes ahead through its own S
// shared-memory slots (ring[slot * blockDim.x + threadIdx.x]) by 8-byte
// cp.async, one commit group per node, so the bytes in flight do not cost
// registers; S = 0 keeps U = 8 nodes ahead in registers.
template <typename T, bool CG, int S = 0>
__device__ __forceinline__ void scan_freq(const ScanParams<T>& p, int l, long long i, unsigned nblk,
                                          cx<T>* ring = nullptr) {
    typedef cx<T> C;
    static_assert(S == 0 || sizeof(T) == 4, "staged node reads of complex64");
    const long long lo = (long long)l * p.N;
    cx<T>* psi = p.psi + lo * (p.M + 1);
    // i: position in the node buffers; k: the frequency there (natural order)
    const long long k = p.tile_logG > 0 ? tile_to_natural(i, p.tile_logG, p.tile_logL, p.N) : i;
    const C zero = mkc(T(0), T(0));
    const C v0 = MPA_DBG_OK(p.dbg, psi + i, sizeof(C)) ? ldx<CG>(psi + i) : zero;
    T rx = T(0.5) * v0.x, ry = T(0.5) * v0.y, cxx = T(0), cyy = T(0);
    const C p0 = MPA_DBG_OK(p.dbg, p.psi0c + lo + k, sizeof(C)) ? ldx<CG>(p.psi0c + lo + k) : zero;
    C vl = v0;
    // node j: psi^{(n+1)}_j = psi_0 + i (R + V_j/2), then R += V_j (Kahan in FP32)
    auto node = [&](int j) {
        if (p.mode == 0) {
            const T sx = (rx - cxx) + T(0.5) * vl.x, sy = (ry - cyy) + T(0.5) * vl.y;
            if (MPA_DBG_OK(p.dbg, psi + (long long)j * p.N + i, sizeof(C))) psi[(long long)j * p.N + i] = mkc(p0.x - sy, p0.y + sx);
        }
        if constexpr (sizeof(T) == 4) {
            kahan_add(rx, cxx, vl.x);
            kahan_add(ry, cyy, vl.y);
        } else {
            rx += vl.x;
            ry += vl.y;
        }
    };
    if constexpr (S > 0) {
        // the loads never touch a node the loop has written (they run ahead)
        C* mine = ring + threadIdx.x;
#pragma unroll
        for (int u = 0; u < S; ++u) {
            if (1 + u <= p.M && MPA_DBG_OK(p.dbg, psi + (long long)(1 + u) * p.N + i, sizeof(C)))
                cp_async8(mine + u * blockDim.x, psi + (long long)(1 + u) * p.N + i);
            cp_async_commit();
        }
        for (int j = 1; j <= p.M; ++j) {
            cp_async_wait_group<S - 1>();  // node j's copy has landed
            C* slot = mine + ((j - 1) % S) * blockDim.x;
            vl = *slot;
            node(j);
            // the slot's value is consumed (node() used it): refill it with node j + S
            if (j + S <= p.M && MPA_DBG_OK(p.dbg, psi + (long long)(j + S) * p.N + i, sizeof(C)))
                cp_async8(slot, psi + (long long)(j + S) * p.N + i);
            cp_async_commit();
        }
        cp_async_wait_group<0>();
    } else {
        // V_j are loaded U nodes ahead of their use (more loads in flight per
        // thread; the loads never touch a node the loop has written)
        constexpr int U = 8;
        C nxt[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            nxt[u] = (1 + u <= p.M && MPA_DBG_OK(p.dbg, psi + (long long)(1 + u) * p.N + i, sizeof(C)))
                         ? ldx<CG>(psi + (long long)(1 + u) * p.N + i)
                         : zero;
        for (int jb = 1; jb <= p.M; jb += U) {
            C cur[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                cur[u] = nxt[u];
                const int jn = jb + U + u;
                nxt[u] = (jn <= p.M && MPA_DBG_OK(p.dbg, psi + (long long)jn * p.N + i, sizeof(C)))
                             ? ldx<CG>(psi + (long long)jn * p.N + i)
                             : zero;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = jb + u;
                if (j > p.M) break;
                vl = cur[u];
                node(j);
            }
        }
    }
    // D = R_M - V_M/2 at node M in FP64 (psi_M = psi_0 + i D)
    const double sx = ((double)rx - (double)cxx) - 0.5 * (double)vl.x;
    const double sy = ((double)ry - (double)cyy) - 0.5 * (double)vl.y;
    if (p.conv) {
        // Picard increment at node M against the previous level's D
        double dx = sx, dy = sy;
        if (p.level > 0) {
            const float2 d0 = MPA_DBG_OK(p.dbg, p.dprev + lo + i, sizeof(float2)) ? ldx<CG>(p.dprev + lo + i)
                                                                                 : make_float2(0.f, 0.f);
            dx -= (double)d0.x;
            dy -= (double)d0.y;
        }
        if (p.level < p.n_iter - 1 && MPA_DBG_OK(p.dbg, p.dprev + lo + i, sizeof(float2)))
            p.dprev[lo + i] = make_float2((float)sx, (float)sy);
        const double px = (double)p0.x - sy, py = (double)p0.y + sx;
        conv_close(p.conv + l, p.err, dx * dx + dy * dy, px * px + py * py, p.level, p.n_iter - 1, p.floor_rel, nblk);
    }
    if (p.mode == 0) return;
    const double2 s0 = MPA_DBG_OK(p.dbg, p.state + lo + k, sizeof(double2)) ? ldx<CG>(p.state + lo + k)
                                                                          : make_double2(0.0, 0.0);
    const double2 psiM = make_double2(s0.x - sy, s0.y + sx);
    if (p.mode == 2) {
        p.out[lo + k] = psiM;  // the caller's buffer (mpa_interval), outside the workspace
        return;
    }
    // step 7 and the lumped gain
    NodeC nodeM{};
    if (MPA_DBG_OK(p.dbg, p.loff + l, sizeof(int)) && MPA_DBG_OK(p.dbg, p.nodes + p.loff[l] + p.M, sizeof(NodeC)))
        nodeM = p.nodes[p.loff[l] + p.M];
    const double2 ph = expi_turns<double>(phase_q64(signed_k(k, p.N), nodeM));
    const double g = nodeM.pre * (MPA_DBG_OK(p.dbg, p.gain + l, sizeof(double)) ? p.gain[l] : 0.0);
    const double2 a = make_double2(g * (psiM.x * ph.x - psiM.y * ph.y), g * (psiM.x * ph.y + psiM.y * ph.x));
    if (MPA_DBG_OK(p.dbg, p.state + lo + k, sizeof(double2))) p.state[lo + k] = a;
    if (MPA_DBG_OK(p.dbg, p.psi0c_out + lo + k, sizeof(C))) p.psi0c_out[lo + k] = mkc((T)a.x, (T)a.y);
    if (!(isfinite(a.x) && isfinite(a.y))) atomicOr(p.err, ERR_NONFINITE);
}

// Nodes in flight per thread of the FP32 scan (shared-memory slots; 0: the
// register form).  Measured on the 2^20 link (126 nodes): 8 slots 31.6 ms
// per 100 km (6.07 TB/s), 16 slots 34.8 ms (fewer resident blocks), the
// register form (8 nodes ahead) 34.0 ms.
#ifndef MPA_SCAN_STAGES
#define MPA_SCAN_STAGES 8
#endif
template <typename T>
__global__ void __launch_bounds__(256) scan_kernel(const ScanParams<T> p) {
    if constexpr (sizeof(T) == 4 && MPA_SCAN_STAGES > 0) {
        __shared__ float2 ring[MPA_SCAN_STAGES * 256];
        scan_freq<T, false, MPA_SCAN_STAGES>(p, blockIdx.y, (long long)blockIdx.x * blockDim.x + threadIdx.x, gridDim.x,
                                             ring);
    } else {
        scan_freq<T, false>(p, blockIdx.y, (long long)blockIdx.x * blockDim.x + threadIdx.x, gridDim.x);
    }
}

// out[c][r] = in[r][c] for an R x Cc matrix (32 x 32 tiles).
template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const cx<T>* __restrict__ in, cx<T>* __restrict__ out,
                                                         long long R, long long Cc) {
    __shared__ cx<T> t[32][33];
    const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const long long r = r0 + y, c = c0 + threadIdx.x;
        if (r < R && c < Cc) t[y][threadIdx.x] = in[r * Cc + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const long long c = c0 + y, r = r0 + threadIdx.x;
        if (r < R && c < Cc) out[c * R + r] = t[threadIdx.x][y];
    }
}

// Precision conversions between the FP64 state and working buffers.
template <typename T>
__global__ void __launch_bounds__(256) to_state_kernel(const cx<T>* in, double2* state, cx<T>* copy, long long N) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const cx<T> v = in[k];
    state[k] = make_double2((double)v.x, (double)v.y);
    if (copy) copy[k] = v;
}
template <typename T>
__global__ void __launch_bounds__(256) from_state_kernel(const double2* state, cx<T>* out, long long N) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double2 v = state[k];
    out[k] = mkc((T)v.x, (T)v.y);
}

}  // namespace mpa
