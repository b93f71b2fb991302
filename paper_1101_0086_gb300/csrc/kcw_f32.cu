// Launchers of the wavefront column pass (FP32) and of its step-7 kernel.
#include "launch.h"

namespace mpa {

// Step 7 after a wavefront interval: A_hat(z0+L) = (psi_0 + i D) exp(i beta_M + int G) * gain (FP64).
// With out != nullptr only psi_M = psi_0 + i D is written to out.
__global__ void __launch_bounds__(256) reconstruct_kernel(double2* state, float2* psi0c, const double2* D, NodeC nodeM,
                                                          double gain, long long N, unsigned int* err, double2* out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const double2 s0 = state[k], d = D[k];
    const double2 psiM = make_double2(s0.x - d.y, s0.y + d.x);
    if (out) {
        out[k] = psiM;
        return;
    }
    const double2 ph = expi_turns<double>(phase_q64(signed_k(k, N), nodeM));
    const double g = nodeM.pre * gain;
    const double2 a = make_double2(g * (psiM.x * ph.x - psiM.y * ph.y), g * (psiM.x * ph.y + psiM.y * ph.x));
    state[k] = a;
    psi0c[k] = make_float2((float)a.x, (float)a.y);
    if (!(isfinite(a.x) && isfinite(a.y))) atomicOr(err, 1u);
}


template <int L>
static cudaError_t kcw_one(const KCWParams& p, int n_tiles, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    typedef KCWGeom<L> Gm;
    static AttrOnce once;
    const cudaError_t ea = attrs_once(once, [] {
        cudaError_t e = cudaFuncSetAttribute(kcw_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Gm::smem_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kcw_kernel<L>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    });
    if (ea != cudaSuccess) return ea;
    const bool prof = g_prof_on.load(std::memory_order_relaxed);
    if (prof) prof_begin(st);
    kcw_kernel<L><<<dim3((unsigned)n_tiles, (unsigned)p.n_jobs), Gm::NT, Gm::smem_bytes, st>>>(p);
    if (prof) {
        // algorithmic bytes: every node of every job read once and (unless it
        // is a last-level node without a successor) written once, plus the
        // running sums in and out and psi_0 read once per node
        double b = 0.0;
        for (int i = 0; i < p.n_jobs; ++i) {
            const KCWJob& j = p.job[i];
            const int written = j.last ? j.n_head : j.n_nodes;
            b += (double)(j.n_nodes + written) * p.N * sizeof(float2) + 4.0 * p.N * sizeof(float2) +
                 (double)j.n_nodes * p.N * sizeof(float2);
        }
        prof_end(PK_KCW, st, b);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t kcw_launch(int logL, const KCWParams& p, cudaStream_t st) {
    const int n_tiles = (int)(p.N1 / kcw_tile_cols(logL));
    switch (logL) {
        case 7: return kcw_one<128>(p, n_tiles, st);
        case 8: return kcw_one<256>(p, n_tiles, st);
        case 9: return kcw_one<512>(p, n_tiles, st);
        case 10: return kcw_one<1024>(p, n_tiles, st);
        case 11: return kcw_one<2048>(p, n_tiles, st);
    }
    return cudaErrorInvalidValue;
}

int kcw_tile_cols(int logL) {
    switch (logL) {
        case 7: return KCWGeom<128>::G;
        case 8: return KCWGeom<256>::G;
        case 9: return KCWGeom<512>::G;
        case 10: return KCWGeom<1024>::G;
        case 11: return KCWGeom<2048>::G;
    }
    return 1 << 30;
}

cudaError_t reconstruct_launch(double2* state, float2* psi0c, const double2* D, const NodeC& nodeM, double gain,
                               long long N, unsigned int* err, double2* out, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    reconstruct_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(state, psi0c, D, nodeM, gain, N, err, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mpa
