// Kernels of the reverse mode of one MPA interval (the adjoint of MPA steps
// 2-7, Eq. (6)), for the gradient of a real loss l.  A gradient g of a
// complex quantity x is dl/dRe x + i dl/dIm x (dl = Re(conj(g) dx)).
//
// Reverse of one level n, node j (forward: P = psi_j e^{i beta_j} pre_j,
// A = F^-1[P], U = |A|^2 A, V_j = sigma_j dz F[U] e^{-i beta_j} / pre_j):
//   KCA_G (column pass)  g_V_j  -> q = e^{+i beta_j} (dz / pre_j) g_V_j -> inverse column DFT
//                        and the beta2 term sum_k (w_k^2/2) Im(conj(g_V) V)
//   KRA (row pass)       A(t), kept by the forward recompute (KR_MPA_KEEP); the inverse
//                        row DFT of g: g_U' = unnormalised (the gradient of U over
//                        sigma_j, F^H = N F^-1);
//                        g_A = sigma_j (2 |A|^2 g_U' + A^2 conj(g_U')) -> forward row DFT,
//                        and the sigma term Re sum_n conj(g_U') U
//   KCA_P (column pass)  forward column DFT -> g_psi_j = e^{-i beta_j} (pre_j / N) F[g_A]
//                        and the beta2 term -sum_k (w_k^2/2) Im(conj(g_psi) psi)
//   RSCAN                step 5 reversed: g_V_j = -i (w_j sum_{l>j} g_psi_l + [j>0] g_psi_j / 2),
//                        w_0 = 1/2, w_j = 1; every g_psi_l also adds to the gradient of psi_0.
//                        Its top form starts from the gradient of the interval output
//                        (step 7 and the gain reversed) and adds that step's beta2 term.
// Each tile of a column or row pass lies inside one node (the plan checks
// G <= N1 and G <= N2), so every tile leaves one partial sum per reduction.
#pragma once

#include "kernels.cuh"

// CTAs per SM the reverse passes are compiled for (1: up to 255 registers,
// no spills; 2: 128 registers, a few spills): 2 for both, measured faster
// (MPA reverse column passes 3.10 -> 3.99 TB/s, row pass 2.36 -> 2.81 TB/s).
#ifndef MPA_ADJ_MINB
#define MPA_ADJ_MINB 2
#endif
#ifndef MPA_ADJ_MINB_R
#define MPA_ADJ_MINB_R 2
#endif

namespace mpa {

enum { KCA_G = 0, KCA_P = 1 };
enum { RSCAN_LEVEL = 0, RSCAN_TOP = 1, RSCAN_SUM = 2 };

// Per-node constants of the reverse pass: dz / exp(int_{z0}^{z_j} G) and sigma(z_j).
struct AdjC {
    double dzp;
    double sig;
};

template <typename T> struct KCAParams {
    cx<T>* g;              // node j at g + j N, in/out
    const cx<T>* aux;      // KCA_G: V_j; KCA_P: psi_j; node j at aux + j aux_stride
    long long aux_stride;  // 0: every node reads aux
    long long N;
    int logN;
    int N1, logN1;
    long long ncols;       // (M+1) N1
    const NodeC* nodes;    // this interval's node constants
    const AdjC* adj;
    double wscale;         // (2 pi / T)^2 / 2
    double* part;          // one partial sum per tile
};

template <typename T> struct KRAParams {
    const cx<T>* a;  // A(t) of the level's nodes, rows as the forward row pass kept them
    cx<T>* g;        // rows after KCA_G; overwritten with the forward row pass of g_A
    long long nrows;
    long long N;
    int logN;
    int N2;
    const AdjC* adj;
    double* part;
};

template <typename T> struct RScanParams {
    cx<T>* g;            // (M+1) x N
    double2* gs0;        // gradient of psi_0 (accumulated)
    long long N;
    int M;
    int mode;
    const double2* gX;   // RSCAN_TOP: gradient of the interval output
    const double2* X;    // RSCAN_TOP: the interval output
    NodeC nodeM;         // RSCAN_TOP: step-7 phase
    double scaleM;       // RSCAN_TOP: exp(-gamma L) times the gain
    double wscale;
    double* part;        // RSCAN_TOP: one partial sum per block
};

// Sum of v over the block (every thread passes its value; the result is
// valid in thread 0).
template <int NT> __device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) s += red[i];
    }
    return s;
}

// Im(conj(a) b)
template <typename C> __device__ __forceinline__ auto im_conj_mul(C a, C b) { return a.x * b.y - a.y * b.x; }

// A thread's partial sum of a reduction: compensated in FP32 (FP64 adds
// are scarce on this GPU), plain in FP64; the block sums it in FP64.
template <typename T> struct PartSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T v) {
        if constexpr (sizeof(T) == 4) kahan_add(s, c, v);
        else s += v;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// k'^2 in the working precision (exact in FP32 up to |k'| = 2^12, then
// rounded once)
template <typename T> __device__ __forceinline__ T ksq(long long kk) {
    const T x = (T)(int)kk;
    return x * x;
}

template <typename T, int L, int MODE>
__global__ void __launch_bounds__(KCGeom<T, L>::NT, KCGeom<T, L>::NT <= 256 ? MPA_ADJ_MINB : 1) kca_kernel(const KCAParams<T> p) {
    typedef cx<T> C;
    typedef KCGeom<T, L> Gm;
    typedef Tiling<T> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    constexpr bool INV = (MODE == KCA_G);
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_COL, P::PSH, true> XF;
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_COL, P::PSH, false> XI;
    typedef typename std::conditional<INV, XI, XF>::type XA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;
    C* ohi = olo + G * Gm::OLO;
    const int tid = threadIdx.x;
    const long long col0 = (long long)blockIdx.x * G;
    const int N1m = p.N1 - 1;
    constexpr bool FAST = sizeof(T) == 4;
    const int node = (int)(col0 >> p.logN1);
    const NodeC nc = p.nodes[node];
    const AdjC ac = p.adj[node];
    const C* aux = p.aux + (long long)node * p.aux_stride;
    C* gn = p.g + (long long)node * p.N;

    tw_init<T, L>(thi, tlo, tid, NT);
    if constexpr (INV) {
        for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
            const int g = i % G, m = i / G;
            const long long k1 = (col0 + g) & N1m;
            if (m < Gm::OLO) olo[m * G + g] = expi_ratio<T>(-k1 * m, p.logN);
            else ohi[(m - Gm::OLO) * G + g] = expi_ratio<T>(-k1 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
        }
    }
    __syncthreads();

    PartSum<T> acc;
    C vin[XA::Q0][XA::R0];
#pragma unroll
    for (int q = 0; q < XA::Q0; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, XA::R0>(tid + q * NT, j, g);
        const long long c = (col0 + g) & N1m;
        // FP32 phases streamed in the order of their finite differences:
        // s = -R0/2 .. R0/2-1, element r = (s + R0) mod R0 (no phase array held)
        const long long D = (long long)p.N1 * (L / XA::R0);
        PhaseRun pr(c + (long long)j * p.N1 - (long long)(XA::R0 / 2) * D, D, nc);
#pragma unroll
        for (int u = 0; u < XA::R0; ++u) {
            const int r = (u + XA::R0 / 2) % XA::R0;
            const long long idx = c + (long long)(j + r * (L / XA::R0)) * p.N1;
            C v = gn[idx];
            if constexpr (INV) {
                const long long kk = signed_k(idx, p.N);
                acc.add(ksq<T>(kk) * im_conj_mul(v, aux[idx]));
                C ph;
                if constexpr (FAST) ph = expi_turns_poly(pr.next());
                else ph = expi_turns<T>(phase_q64(kk, nc));
                v = cscale(cmul(v, ph), (T)ac.dzp);
            }
            vin[q][r] = v;
        }
    }

    C vout[XA::QL][XA::RL];
    XA::run(vin, vout, s, thi, tlo);

    const T post = (T)(nc.pre / (double)p.N);
#pragma unroll
    for (int q = 0; q < XA::QL; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, XA::RL>(tid + q * NT, j, g);
        const long long c = (col0 + g) & N1m;
        const long long D = (long long)p.N1 * (L / XA::RL);
        PhaseRun pr(c + (long long)j * p.N1 - (long long)(XA::RL / 2) * D, D, nc);
        constexpr bool HOIST = (L / XA::RL) % Gm::OLO == 0;  // one low-table lookup per butterfly
        C wlo = mkc(T(1), T(0));
        if constexpr (INV && HOIST) wlo = olo[(j & (Gm::OLO - 1)) * G + g];
#pragma unroll
        for (int u = 0; u < XA::RL; ++u) {
            const int r = (u + XA::RL / 2) % XA::RL;  // the phase order, as in the load
            const int row = j + r * (L / XA::RL);
            const long long idx = c + (long long)row * p.N1;
            C v = vout[q][r];
            if constexpr (INV) {
                C w = HOIST ? wlo : olo[(row & (Gm::OLO - 1)) * G + g];
                if constexpr (Gm::OHI > 1) w = cmul(ohi[(row >> Gm::OSH) * G + g], w);
                v = cmul(v, w);
            } else {
                const long long kk = signed_k(idx, p.N);
                C ph;
                if constexpr (FAST) ph = expi_turns_poly(pr.next());
                else ph = expi_turns<T>(phase_q64(kk, nc));
                v = cscale(cmul(v, cconj(ph)), post);
                acc.add(-ksq<T>(kk) * im_conj_mul(v, aux[idx]));
            }
            gn[idx] = v;
        }
    }
    const double tot = block_sum<NT>(acc.value(), red);
    if (tid == 0) p.part[blockIdx.x] = tot * p.wscale;
}

template <typename T, int L>
__global__ void __launch_bounds__(KRGeom<T, L>::NT, KRGeom<T, L>::NT <= 256 ? MPA_ADJ_MINB_R : 1) kra_kernel(const KRAParams<T> p) {
    typedef cx<T> C;
    typedef KRGeom<T, L> Gm;
    typedef Tiling<T, 1> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_ROW, P::PSH, false> XI;
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_ROW, P::PSH, true> XF;
    static_assert(XI::RL == XF::R0, "inverse/forward junction radix");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;
    C* ohi = olo + G * Gm::OLO;
    const int tid = threadIdx.x;
    const long long row0 = (long long)blockIdx.x * G;
    const T sig = (T)p.adj[row0 / p.N2].sig;

    tw_init<T, L>(thi, tlo, tid, NT);
    for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
        const int g = i / (Gm::OLO + Gm::OHI), m = i % (Gm::OLO + Gm::OHI);
        const long long n2 = (row0 + g) & (p.N2 - 1);
        if (m < Gm::OLO) olo[g * Gm::OLO + m] = expi_ratio<T>(n2 * m, p.logN);
        else ohi[g * Gm::OHI + (m - Gm::OLO)] = expi_ratio<T>(n2 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
    }
    __syncthreads();

    // the unnormalised inverse of q, on the element layout in which the
    // forward row pass kept A(t)
    C vg[XI::QL][XI::RL];
    {
        C vin[XI::Q0][XI::R0];
#pragma unroll
        for (int q = 0; q < XI::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_ROW, L, G, XI::R0>(tid + q * NT, j, g);
            const C* src = p.g + (row0 + g) * L;
#pragma unroll
            for (int r = 0; r < XI::R0; ++r) vin[q][r] = src[j + r * (L / XI::R0)];
        }
        XI::run(vin, vg, s, thi, tlo);
    }
    PartSum<T> acc;
#pragma unroll
    for (int q = 0; q < XI::QL; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XI::RL>(tid + q * NT, j, g);
        const C* at = p.a + (row0 + g) * L;
#pragma unroll
        for (int r = 0; r < XI::RL; ++r) {
            const C a = at[j + r * (L / XI::RL)];
            const C gu = vg[q][r];
            const T pw = a.x * a.x + a.y * a.y;
            acc.add(pw * (gu.x * a.x + gu.y * a.y));  // Re(conj(g_U') U)
            const C a2 = mkc(a.x * a.x - a.y * a.y, T(2) * a.x * a.y);
            const C t = cmul(a2, cconj(gu));
            vg[q][r] = mkc(sig * (T(2) * pw * gu.x + t.x), sig * (T(2) * pw * gu.y + t.y));
        }
    }
    C vout[XF::QL][XF::RL];
    XF::run(vg, vout, s, thi, tlo);
#pragma unroll
    for (int q = 0; q < XF::QL; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XF::RL>(tid + q * NT, j, g);
        C* dst = p.g + (row0 + g) * L;
        constexpr bool HOIST = (L / XF::RL) % Gm::OLO == 0;
        const C wlo = HOIST ? olo[g * Gm::OLO + (j & (Gm::OLO - 1))] : mkc(T(1), T(0));
#pragma unroll
        for (int r = 0; r < XF::RL; ++r) {
            const int l = j + r * (L / XF::RL);
            C w = HOIST ? wlo : olo[g * Gm::OLO + (l & (Gm::OLO - 1))];
            if constexpr (Gm::OHI > 1) w = cmul(ohi[g * Gm::OHI + (l >> Gm::OSH)], w);
            dst[l] = cmul(vout[q][r], w);
        }
    }
    const double tot = block_sum<NT>(acc.value(), red);
    if (tid == 0) p.part[blockIdx.x] = tot;
}

// Step 5 reversed for every frequency (see the header comment), and its
// top and closing forms.
template <typename T>
__global__ void __launch_bounds__(256) rscan_kernel(const RScanParams<T> p) {
    typedef cx<T> C;
    __shared__ double red[8];
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (k < p.N) {
        C* g = p.g;
        if (p.mode == RSCAN_TOP) {
            // A_hat(z0+L) = psi_M e^{i beta_M} pre_M gain: g_psi_M = conj(e^{i beta_M} pre_M gain) g_X
            const long long kk = signed_k(k, p.N);
            const double2 ph = expi_turns<double>(phase_q64(kk, p.nodeM));
            const double2 gx = p.gX[k], x = p.X[k];
            const double2 gm = make_double2(p.scaleM * (ph.x * gx.x + ph.y * gx.y),
                                            p.scaleM * (ph.x * gx.y - ph.y * gx.x));
            acc = -(double)(kk * kk) * (gx.x * x.y - gx.y * x.x);
            double2 s0 = p.gs0[k];
            p.gs0[k] = make_double2(s0.x + gm.x, s0.y + gm.y);
            // g_V_j = -i w_j g_psi_M with w_0 = w_M = 1/2
            const C full = mkc((T)gm.y, (T)(-gm.x)), half = mkc((T)(0.5 * gm.y), (T)(-0.5 * gm.x));
            g[k] = half;
            for (int j = 1; j < p.M; ++j) g[(long long)j * p.N + k] = full;
            g[(long long)p.M * p.N + k] = half;
        } else if (p.mode == RSCAN_LEVEL) {
            T tx = T(0), ty = T(0), cx_ = T(0), cy_ = T(0);  // sum_{l>j} g_psi_l (compensated in FP32)
            // sum over all l for the gradient of psi_0: compensated in the
            // working precision (FP64 adds are scarce on this GPU)
            T sx = T(0), sy = T(0), csx = T(0), csy = T(0);
            // nodes loaded U ahead of their use (downwards; never a node already written)
            constexpr int U = 8;
            C nxt[U];
#pragma unroll
            for (int u = 0; u < U; ++u) nxt[u] = (p.M - u >= 0) ? g[(long long)(p.M - u) * p.N + k] : mkc(T(0), T(0));
            for (int jb = p.M; jb >= 0; jb -= U) {
                C cur[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    cur[u] = nxt[u];
                    const int jn = jb - U - u;
                    nxt[u] = (jn >= 0) ? g[(long long)jn * p.N + k] : mkc(T(0), T(0));
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = jb - u;
                    if (j < 0) break;
                    const C gl = cur[u];
                    if constexpr (sizeof(T) == 4) {
                        kahan_add(sx, csx, gl.x);
                        kahan_add(sy, csy, gl.y);
                    } else {
                        sx += gl.x;
                        sy += gl.y;
                    }
                    const T ux = tx - cx_, uy = ty - cy_;
                    const T ax = j == 0 ? T(0.5) * ux : ux + T(0.5) * gl.x;
                    const T ay = j == 0 ? T(0.5) * uy : uy + T(0.5) * gl.y;
                    g[(long long)j * p.N + k] = mkc(ay, -ax);
                    if (j > 0) {
                        if constexpr (sizeof(T) == 4) {
                            kahan_add(tx, cx_, gl.x);
                            kahan_add(ty, cy_, gl.y);
                        } else {
                            tx += gl.x;
                            ty += gl.y;
                        }
                    }
                }
            }
            double2 s0 = p.gs0[k];
            p.gs0[k] = make_double2(s0.x + ((double)sx - (double)csx), s0.y + ((double)sy - (double)csy));
        } else {
            T sx = T(0), sy = T(0), csx = T(0), csy = T(0);
            constexpr int U = 8;
            for (int jb = 0; jb <= p.M; jb += U) {
                C cur[U];
#pragma unroll
                for (int u = 0; u < U; ++u) cur[u] = (jb + u <= p.M) ? g[(long long)(jb + u) * p.N + k] : mkc(T(0), T(0));
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if constexpr (sizeof(T) == 4) {
                        kahan_add(sx, csx, cur[u].x);
                        kahan_add(sy, csy, cur[u].y);
                    } else {
                        sx += cur[u].x;
                        sy += cur[u].y;
                    }
                }
            }
            double2 s0 = p.gs0[k];
            p.gs0[k] = make_double2(s0.x + ((double)sx - (double)csx), s0.y + ((double)sy - (double)csy));
        }
    }
    if (p.mode == RSCAN_TOP) {
        const double tot = block_sum<256>(acc, red);
        if (threadIdx.x == 0) p.part[blockIdx.x] = tot * p.wscale;
    }
}

// Eq. (6) partial sums of one level into a separate buffer (the forward scan
// of level n without step 7), node 0 receiving psi_0: the same arithmetic
// and order as the forward scan, so the recomputed levels equal the
// forward pass's.
template <typename T>
__global__ void __launch_bounds__(256) scan_store_kernel(const cx<T>* __restrict__ v, cx<T>* __restrict__ psi,
                                                         const cx<T>* __restrict__ psi0c, long long N, int M) {
    typedef cx<T> C;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const C v0 = v[k];
    T rx = T(0.5) * v0.x, ry = T(0.5) * v0.y, cxx = T(0), cyy = T(0);
    const C p0 = psi0c[k];
    psi[k] = p0;
    for (int j = 1; j <= M; ++j) {
        const C vl = v[(long long)j * N + k];
        const T sx = (rx - cxx) + T(0.5) * vl.x, sy = (ry - cyy) + T(0.5) * vl.y;
        psi[(long long)j * N + k] = mkc(p0.x - sy, p0.y + sx);
        if constexpr (sizeof(T) == 4) {
            kahan_add(rx, cxx, vl.x);
            kahan_add(ry, cyy, vl.y);
        } else {
            rx += vl.x;
            ry += vl.y;
        }
    }
}

// ---------------------------------------------------------------- split-step
// Reverse mode of the split-step of Eq. (4) on the same four-step layout as
// its forward kernels (kc_kernel KC_SS_STEP, kr_kernel KR_SS).
//   SSC (column pass)  STORE: forward column DFT -> X' = X exp(i beta) pre (kept, natural
//                      order) -> inverse column DFT, exactly as KC_SS_STEP.
//                      REV: forward column DFT -> g; the beta2 term -sum_k (w_k^2/2) Im(conj(g) X')
//                      -> g conj(exp(i beta)) pre -> inverse column DFT.
//   SSR (row pass)     STORE: inverse row DFT -> t = (.)/N (kept) -> t exp(i s |t|^2) -> forward,
//                      exactly as KR_SS.
//                      REV: inverse row DFT -> g~ = (.)/N (the gradient of y over N);
//                      y = t e^{i s |t|^2}, c = -Im(conj(g~) y):
//                      g~_t = e^{-i s |t|^2} g~ + 2 c s t, the sigma term N sum c |t|^2 -> forward.
enum { SS_STORE = 0, SS_REV = 1 };

template <typename T> struct SSCParams {
    cx<T>* data;     // N samples, work layout, in/out
    cx<T>* xs;       // X' of this linear step (natural order): written by STORE, read by REV
    long long N;
    int logN;
    int N1, logN1;
    NodeC flow;      // STORE: exp(i beta) and pre of the step; REV: the negated phase
    double pre;      // the real factor applied (STORE: flow.pre; REV: flow.pre, / N on the output side)
    double wscale;   // (2 pi / T)^2 / 2, times the factor the incoming gradient still lacks (1/N on the output side)
    double* part;
};

template <typename T> struct SSRParams {
    cx<T>* data;  // N1-sample rows, in/out
    cx<T>* ts;    // t of this nonlinear step (work layout): written by STORE, read by REV
    long long nrows;
    long long N;
    int logN;
    int N2;
    T inv_n;
    T rot;        // int sigma over the step
    double scale; // REV: factor of the sigma partial sums (N)
    double* part;
};

template <typename T, int L, int MODE>
__global__ void __launch_bounds__(KCGeom<T, L>::NT, KCGeom<T, L>::NT <= 256 ? MPA_ADJ_MINB : 1) ssc_kernel(const SSCParams<T> p) {
    typedef cx<T> C;
    typedef KCGeom<T, L> Gm;
    typedef Tiling<T> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_COL, P::PSH, true> XF;
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_COL, P::PSH, false> XI;
    static_assert(XF::RL == XI::R0, "forward/inverse junction radix");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;
    C* ohi = olo + G * Gm::OLO;
    const int tid = threadIdx.x;
    const long long col0 = (long long)blockIdx.x * G;
    const int N1m = p.N1 - 1;
    constexpr bool FAST = sizeof(T) == 4;

    tw_init<T, L>(thi, tlo, tid, NT);
    for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
        const int g = i % G, m = i / G;
        const long long k1 = (col0 + g) & N1m;
        if (m < Gm::OLO) olo[m * G + g] = expi_ratio<T>(-k1 * m, p.logN);
        else ohi[(m - Gm::OLO) * G + g] = expi_ratio<T>(-k1 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
    }
    __syncthreads();

    C vin[XF::Q0][XF::R0];
#pragma unroll
    for (int q = 0; q < XF::Q0; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, XF::R0>(tid + q * NT, j, g);
        const long long c = (col0 + g) & N1m;
#pragma unroll
        for (int r = 0; r < XF::R0; ++r) vin[q][r] = p.data[c + (long long)(j + r * (L / XF::R0)) * p.N1];
    }
    C vm[XF::QL][XF::RL];
    XF::run(vin, vm, s, thi, tlo);
    PartSum<T> acc;
#pragma unroll
    for (int q = 0; q < XF::QL; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, XF::RL>(tid + q * NT, j, g);
        const long long c = (col0 + g) & N1m;
        unsigned long long th[XF::RL];
        if constexpr (FAST) phase_run<XF::RL>(c + (long long)j * p.N1, (long long)p.N1 * (L / XF::RL), p.flow, th);
#pragma unroll
        for (int r = 0; r < XF::RL; ++r) {
            const long long idx = c + (long long)(j + r * (L / XF::RL)) * p.N1;
            C ph;
            if constexpr (FAST) ph = expi_turns_poly(th[r]);
            else ph = expi_turns<T>(phase_q64(signed_k(idx, p.N), p.flow));
            if constexpr (MODE == SS_REV) acc.add(-ksq<T>(signed_k(idx, p.N)) * im_conj_mul(vm[q][r], p.xs[idx]));
            vm[q][r] = cscale(cmul(vm[q][r], ph), (T)p.pre);
            if constexpr (MODE == SS_STORE) p.xs[idx] = vm[q][r];
        }
    }
    C vout[XI::QL][XI::RL];
    XI::run(vm, vout, s, thi, tlo);
#pragma unroll
    for (int q = 0; q < XI::QL; ++q) {
        int j, g;
        bmap<LAYOUT_COL, L, G, XI::RL>(tid + q * NT, j, g);
        const long long c = (col0 + g) & N1m;
        constexpr bool HOIST = (L / XI::RL) % Gm::OLO == 0;
        const C wlo = HOIST ? olo[(j & (Gm::OLO - 1)) * G + g] : mkc(T(1), T(0));
#pragma unroll
        for (int r = 0; r < XI::RL; ++r) {
            const int row = j + r * (L / XI::RL);
            C w = HOIST ? wlo : olo[(row & (Gm::OLO - 1)) * G + g];
            if constexpr (Gm::OHI > 1) w = cmul(ohi[(row >> Gm::OSH) * G + g], w);
            p.data[c + (long long)row * p.N1] = cmul(vout[q][r], w);
        }
    }
    if constexpr (MODE == SS_REV) {
        const double tot = block_sum<NT>(acc.value(), red);
        if (tid == 0) p.part[blockIdx.x] = tot * p.wscale;
    }
}

template <typename T, int L, int MODE>
__global__ void __launch_bounds__(KRGeom<T, L>::NT, KRGeom<T, L>::NT <= 256 ? MPA_ADJ_MINB_R : 1) ssr_kernel(const SSRParams<T> p) {
    typedef cx<T> C;
    typedef KRGeom<T, L> Gm;
    typedef Tiling<T, 1> P;
    constexpr int G = Gm::G, TE = Gm::TE, NT = Gm::NT;
    typedef Xform<T, L, G, NT, P::RMAX, -1, LAYOUT_ROW, P::PSH, false> XI;
    typedef Xform<T, L, G, NT, P::RMAX, +1, LAYOUT_ROW, P::PSH, true> XF;
    static_assert(XI::RL == XF::R0, "inverse/forward junction radix");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    C* s = reinterpret_cast<C*>(smem_raw);
    C* thi = s + TE + (TE >> P::PSH) + 1;
    C* tlo = thi + TwDims<L>::NHI;
    C* olo = tlo + TwDims<L>::NLO;
    C* ohi = olo + G * Gm::OLO;
    const int tid = threadIdx.x;
    const long long row0 = (long long)blockIdx.x * G;

    tw_init<T, L>(thi, tlo, tid, NT);
    for (int i = tid; i < G * (Gm::OLO + Gm::OHI); i += NT) {
        const int g = i / (Gm::OLO + Gm::OHI), m = i % (Gm::OLO + Gm::OHI);
        const long long n2 = (row0 + g) & (p.N2 - 1);
        if (m < Gm::OLO) olo[g * Gm::OLO + m] = expi_ratio<T>(n2 * m, p.logN);
        else ohi[g * Gm::OHI + (m - Gm::OLO)] = expi_ratio<T>(n2 * ((long long)(m - Gm::OLO) << Gm::OSH), p.logN);
    }
    __syncthreads();

    C vin[XI::Q0][XI::R0];
#pragma unroll
    for (int q = 0; q < XI::Q0; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XI::R0>(tid + q * NT, j, g);
        const C* src = p.data + (row0 + g) * L;
#pragma unroll
        for (int r = 0; r < XI::R0; ++r) vin[q][r] = src[j + r * (L / XI::R0)];
    }
    C vm[XI::QL][XI::RL];
    XI::run(vin, vm, s, thi, tlo);
    PartSum<T> acc;
#pragma unroll
    for (int q = 0; q < XI::QL; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XI::RL>(tid + q * NT, j, g);
        C* tr = p.ts + (row0 + g) * L;
#pragma unroll
        for (int r = 0; r < XI::RL; ++r) {
            const int l = j + r * (L / XI::RL);
            if constexpr (MODE == SS_STORE) {
                C a = cscale(vm[q][r], p.inv_n);
                tr[l] = a;
                const T pw = a.x * a.x + a.y * a.y;
                T sn, cs;
                sincos_kerr(p.rot * pw, &sn, &cs);
                vm[q][r] = cmul(a, mkc(cs, sn));
            } else {
                const C gy = cscale(vm[q][r], p.inv_n);
                const C t = tr[l];
                const T pw = t.x * t.x + t.y * t.y;
                T sn, cs;
                sincos_kerr(p.rot * pw, &sn, &cs);
                const C e = mkc(cs, sn);
                const C y = cmul(t, e);
                const T c = -im_conj_mul(gy, y);
                acc.add(c * pw);
                const C a = cmul(gy, cconj(e));
                const T f = T(2) * c * p.rot;
                vm[q][r] = mkc(a.x + f * t.x, a.y + f * t.y);
            }
        }
    }
    C vout[XF::QL][XF::RL];
    XF::run(vm, vout, s, thi, tlo);
#pragma unroll
    for (int q = 0; q < XF::QL; ++q) {
        int j, g;
        bmap<LAYOUT_ROW, L, G, XF::RL>(tid + q * NT, j, g);
        C* dst = p.data + (row0 + g) * L;
        constexpr bool HOIST = (L / XF::RL) % Gm::OLO == 0;
        const C wlo = HOIST ? olo[g * Gm::OLO + (j & (Gm::OLO - 1))] : mkc(T(1), T(0));
#pragma unroll
        for (int r = 0; r < XF::RL; ++r) {
            const int l = j + r * (L / XF::RL);
            C w = HOIST ? wlo : olo[g * Gm::OLO + (l & (Gm::OLO - 1))];
            if constexpr (Gm::OHI > 1) w = cmul(ohi[g * Gm::OHI + (l >> Gm::OSH)], w);
            dst[l] = cmul(vout[q][r], w);
        }
    }
    if constexpr (MODE == SS_REV) {
        const double tot = block_sum<NT>(acc.value(), red);
        if (tid == 0) p.part[blockIdx.x] = tot * p.scale;
    }
}

// state = scale * in (FP64).
template <typename T>
__global__ void __launch_bounds__(256) scale_to_state_kernel(const cx<T>* in, double2* state, double scale,
                                                             long long N) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const cx<T> v = in[k];
    state[k] = make_double2(scale * (double)v.x, scale * (double)v.y);
}

}  // namespace mpa
