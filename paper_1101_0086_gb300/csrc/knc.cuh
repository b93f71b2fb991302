// The on-chip node transform for N = C x 2^14 FP32 modes (C = 2, 4): one
// thread-block cluster of C CTAs per node, each holding a 2^14-sample slice
// in its shared memory and reading its partners' slices through distributed
// shared memory (no multicast, no global round trip).
//
// With N = C P, k = p + P r (CTA r holds the natural-order slice
// [r P, r P + P)) and n = C q + m, the inverse transform of MPA step 3,
//   A(C q + m) = (1/N) sum_p W_P^{-q p} W_N^{-m p} sum_r W_C^{-m r} A_hat(p + P r),
// is a length-C DFT across the cluster (CTA m keeps output m), the factor
// W_N^{-m p} and a length-P transform inside CTA m, which then holds the
// samples n = m (mod C).  |A|^2 A is pointwise.  The forward transform of
// step 4 mirrors it:
//   V(p + P r) = sum_m W_C^{m r} W_N^{m p} sum_q W_P^{q p} U(C q + m).
// The phases exp(+-i beta_j) and the Eq. (6) weight are applied at the load
// and the store as in kn_kernel.  Every CTA of a cluster passes the same four
// cluster barriers (hardware barriers; no CTA leaves early).
#pragma once

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace mpa {

template <int C> struct KNCGeom {
    static constexpr int P = 16384, NT = 512;
    typedef Tiling<float, 1> Pt;  // 32 elements per thread, radix 32
    static constexpr size_t smem_bytes =
        ((size_t)P + (P >> Pt::PSH) + 1 + TwDims<P>::NLO + TwDims<P>::NHI + 2 * 128) * sizeof(float2);
};

// x * W_C^{S e} for e = 0 .. C-1 (C = 2 or 4): multiplications by +-1, +-i
template <int C, int S> __device__ __forceinline__ float2 rot_c(float2 x, int e) {
    if constexpr (C == 2) {
        return (e & 1) ? make_float2(-x.x, -x.y) : x;
    } else {
        switch (e & 3) {
            case 0: return x;
            case 1: return mul_si<S>(x);
            case 2: return make_float2(-x.x, -x.y);
            default: return mul_si<-S>(x);
        }
    }
}

// Shared-memory address (32-bit, shared::cluster window) of the same offset
// in the shared memory of CTA `rank` of the cluster, and a load from it.
__device__ __forceinline__ unsigned cluster_smem_addr(const void* local, unsigned rank) {
    const unsigned la = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    return ra;
}
template <unsigned OFF> __device__ __forceinline__ float2 ld_cluster_f2(unsigned addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(OFF));
    return v;
}

// The length-C DFT across the cluster for this thread's 32 elements
// pp = tid + 512 r (padded slot tid + tid/32 + 528 r, so element r sits at a
// compile-time byte offset 4224 r from the thread's base): out[r] =
// sum_c W_C^{S m c} x_c(pp) with x_c read from CTA c.  The offsets go into
// the load instructions as immediates, so no per-element address registers.
template <int C, int S, int R>
__device__ __forceinline__ void cluster_dft_rows(float2 (&out)[32], const unsigned (&rs)[C], int m) {
    if constexpr (R < 32) {
        constexpr unsigned OFF = (unsigned)R * 4224u;
        float2 acc = ld_cluster_f2<OFF>(rs[0]);
#pragma unroll
        for (int c = 1; c < C; ++c) acc = cadd(acc, rot_c<C, S>(ld_cluster_f2<OFF>(rs[c]), m * c));
        out[R] = acc;
        cluster_dft_rows<C, S, R + 1>(out, rs, m);
    }
}

template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(512, 1) knc_kernel(const KNParams<float> p) {
    namespace cg = cooperative_groups;
    typedef KNCGeom<C> Gm;
    typedef typename Gm::Pt Pt;
    constexpr int P = Gm::P, NT = Gm::NT, LOGN = (C == 2 ? 15 : 16);
    typedef Xform<float, P, 1, NT, Pt::RMAX, -1, LAYOUT_ROW, Pt::PSH, false> XI;
    typedef Xform<float, P, 1, NT, Pt::RMAX, +1, LAYOUT_ROW, Pt::PSH, true> XF;
    static_assert(XI::Q0 == 1 && XI::R0 == 32 && XF::QL == 1 && XF::RL == 32, "one 32-element butterfly per thread");
    static_assert(XI::RL == XF::R0, "inverse/forward junction radix");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* s = reinterpret_cast<float2*>(smem_raw);
    float2* thi = s + P + (P >> Pt::PSH) + 1;
    float2* tlo = thi + TwDims<P>::NHI;
    float2* whi = tlo + TwDims<P>::NLO;  // W_N^{m 128 h}
    float2* wlo = whi + 128;              // W_N^{m l}
    cg::cluster_group cl = cg::this_cluster();
    const int m = (int)cl.block_rank();
    const int tid = threadIdx.x;
    const int node = (int)(blockIdx.x / C);  // the grid holds exactly nrows clusters
    // this thread's elements of the slice: pp = tid + 512 r, k = m P + pp;
    // signed k' = k - N on the upper half (whole slices, C even).  The node's
    // constants and pointers are read again after the transforms rather than
    // kept live through them (register pressure).
    const long long kf = (long long)m * P + tid - (m >= C / 2 ? (long long)C * P : 0ll);

    tw_init<float, P>(thi, tlo, tid, NT);
    for (int i = tid; i < 256; i += NT) {
        if (i < 128) whi[i] = expi_ratio<float>((long long)m * ((long long)i << 7), LOGN);
        else wlo[i - 128] = expi_ratio<float>((long long)m * (i - 128), LOGN);
    }
    // ---- step 2 on the slice, into shared memory in natural order
    {
        const int l = node / p.npl, jn = node - l * p.npl;
        const float2* src =
            (p.src0 && jn == 0) ? p.src0 + l * p.src0_lstride : p.src + l * p.src_lstride + jn * p.src_stride;
        const NodeC nc = p.nodes[p.loff[l] + jn];
        PhaseRun pr(kf, 512, nc);
        const float pre = (float)nc.pre;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int pp = tid + 512 * r;
            const float2 v = src[(long long)m * P + pp];
            s[phys<Pt::PSH>(pp)] = cscale(cmul(v, expi_turns_poly(pr.next())), pre);
        }
    }
    cl.sync();
    // ---- length-C inverse DFT across the cluster (output m), factor W_N^{-m pp}
    float2 vin[1][32];
    {
        // this thread's slot in each CTA of the cluster (32-bit shared::cluster addresses)
        unsigned rs[C];
#pragma unroll
        for (int c = 0; c < C; ++c) rs[c] = cluster_smem_addr(s + phys<Pt::PSH>(tid), (unsigned)c);
        cluster_dft_rows<C, -1, 0>(vin[0], rs, m);
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int pp = tid + 512 * r;
            vin[0][r] = cmul(vin[0][r], cconj(cmul(whi[pp >> 7], wlo[pp & 127])));
        }
    }
    cl.sync();  // every partner has read this slice before the tile is reused
    // ---- length-P inverse transform, 1/N, |A|^2 A, length-P forward transform
    float2 vm[XI::QL][XI::RL];
    XI::run(vin, vm, s, thi, tlo);
#pragma unroll
    for (int q = 0; q < XI::QL; ++q) {
#pragma unroll
        for (int r = 0; r < XI::RL; ++r) {
            const float2 a = cscale(vm[q][r], p.inv_n);
            vm[q][r] = cscale(a, a.x * a.x + a.y * a.y);
        }
    }
    float2 vout[1][32];
    XF::run(vm, vout, s, thi, tlo);
    // ---- factor W_N^{m pp}, into shared memory for the partners
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int pp = tid + 512 * r;
        s[phys<Pt::PSH>(pp)] = cmul(vout[0][r], cmul(whi[pp >> 7], wlo[pp & 127]));
    }
    cl.sync();
    // ---- length-C forward DFT across the cluster (this CTA's slice m),
    // V_j = F[U] exp(-i beta_j) sigma_j dz / exp(int G)  (Eq. (6))
    {
        const int l = node / p.npl, jn = node - l * p.npl;
        float2* dst = p.dst + l * p.dst_lstride + jn * p.dst_stride;
        const NodeC nc = p.nodes[p.loff[l] + jn];
        unsigned rs[C];
#pragma unroll
        for (int c = 0; c < C; ++c) rs[c] = cluster_smem_addr(s + phys<Pt::PSH>(tid), (unsigned)c);
        cluster_dft_rows<C, +1, 0>(vout[0], rs, m);
        PhaseRun pr(kf, 512, nc);
        const float post = (float)nc.post;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int pp = tid + 512 * r;
            dst[(long long)m * P + pp] = cscale(cmul(vout[0][r], cconj(expi_turns_poly(pr.next()))), post);
        }
    }
    cl.sync();  // keep this slice alive until every partner has read it
}

}  // namespace mpa
