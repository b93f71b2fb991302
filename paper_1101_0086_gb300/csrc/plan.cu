// C ABI of the MPA / split-step library: plan creation (host tables of the
// per-node constants of Eq. (6)), workspace layout, and the launch schedule
// of the MPA steps 1-7 and of the split-step of Eq. (4).
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "adj_launch.h"
#include "plan.h"

using namespace mpa;

namespace mpa {
namespace host {
thread_local std::string g_cuda_err;
int cuda_fail(cudaError_t e) {
    g_cuda_err = cudaGetErrorString(e);
    return MPA_ERR_CUDA;
}
}  // namespace host
}  // namespace mpa

using namespace mpa::host;

namespace mpa {
namespace host {

// One level-synchronous interval for nl links stored link-major (link l's
// node j at psi + (l (M+1) + j) N, its psi_0 at psi0c + l N, its FP64 state
// at state + l N).  loff[l] points link l's node constants for this
// interval; gain[l] is its amplifier gain at the interval end (device).
// Every iteration covers nodes 0..M of every link; node 0 always reads
// psi_0, so V_0 (identical at every iteration) is simply recomputed.
template <typename T>
int mpa_levels(const Split& s, int M, int n_iter, int nl, cx<T>* psi, cx<T>* work, cx<T>* psi0c, double2* state,
               const NodeC* nodes, const int* loff, const double* gain, const Monitor& mon, int scan_mode,
               double2* out, cudaStream_t st) {
    const long long N = s.N;
    const int npl = M + 1;
    int tile_log_g = 0;  // > 0: node spectra between the passes in the staged column pass's tile layout
    for (int n = 0; n < n_iter; ++n) {
        if (s.onchip) {
            // steps 2-4 and the weight of Eq. (6), one launch for every node of every link
            KNParams<T> k{};
            k.src = n == 0 ? psi0c : psi;
            k.src_stride = n == 0 ? 0 : N;
            k.src_lstride = n == 0 ? N : (long long)npl * N;
            k.src0 = psi0c;
            k.src0_lstride = N;
            k.dst = psi;
            k.dst_stride = N;
            k.dst_lstride = (long long)npl * N;
            k.nrows = (long long)nl * npl;
            k.npl = npl;
            k.nodes = nodes;
            k.loff = loff;
            k.inv_n = (T)(1.0 / (double)N);
            k.dbg = mon.dbg;
            MPA_TRY(kn_launch<T>(s.logN, k, st));
        } else {
        // steps 2-4 at every node (one launch per pass for all links)
        KCParams<T> c{};
        c.src = n == 0 ? psi0c : psi;
        c.src_stride = n == 0 ? 0 : N;
        c.src_lstride = n == 0 ? N : (long long)npl * N;
        c.src0 = psi0c;
        c.src0_lstride = N;
        c.dst = psi;
        c.dst_stride = N;
        c.dst_lstride = (long long)npl * N;
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.ncols = (long long)nl * npl * s.N1;
        c.npl = npl;
        c.nodes = nodes;
        c.loff = loff;
        c.err = mon.err;
        c.spin_limit = mon.spin_limit;
        c.dbg = mon.dbg;
        if constexpr (sizeof(T) == 4)
            tile_log_g = work && kc_staged(KC_MPA_POST, s.logN2, c) ? kcs_tile_log_cols(s.logN2) : 0;
        // Tile layout: the forward pass writes V_j into psi in the tile layout
        // of the staged column pass, the scan keeps it for psi^{(n+1)}, and the
        // next inverse pass reads whole tiles from psi and writes the natural
        // order into `work`, where the row pass and the forward pass run.
        cx<T>* xw = tile_log_g > 0 ? work : psi;
        c.tiled_in = n > 0 && tile_log_g > 0;
        c.dst = xw;
        MPA_TRY(kc_launch<T>(KC_MPA_PRE, s.logN2, c, st));
        KRParams<T> r{xw, (long long)nl * npl * s.N2, N, s.logN, (int)s.N2, (T)(1.0 / (double)N), T(0)};
        r.err = mon.err;
        r.spin_limit = mon.spin_limit;
        r.dbg = mon.dbg;
        MPA_TRY(kr_launch<T>(KR_MPA, s.logN1, r, st));
        c.src = xw;
        c.src_stride = N;
        c.src_lstride = (long long)npl * N;
        c.src0 = nullptr;
        c.dst = psi;
        c.tiled_in = 0;
        c.tiled_out = tile_log_g > 0;
        MPA_TRY(kc_launch<T>(KC_MPA_POST, s.logN2, c, st));
        }
        // step 5 (Eq. (6)); on the last iteration fused with step 7
        ScanParams<T> q{};
        q.psi = psi;
        q.N = N;
        q.M = M;
        q.psi0c = psi0c;
        q.state = state;
        q.psi0c_out = psi0c;
        q.out = out;
        q.mode = (n == n_iter - 1) ? scan_mode : 0;
        q.nodes = nodes;
        q.loff = loff;
        q.gain = gain;
        q.err = mon.err;
        q.conv = mon.conv;
        q.dprev = mon.dprev;
        q.level = n;
        q.n_iter = n_iter;
        q.floor_rel = kDivergenceFloor;
        q.tile_logG = tile_log_g;
        q.tile_logL = s.logN2;
        q.dbg = mon.dbg;
        MPA_TRY(scan_launch<T>(q, nl, st));
    }
    return MPA_OK;
}

template int mpa_levels<float>(const Split&, int, int, int, float2*, float2*, float2*, double2*, const NodeC*,
                               const int*, const double*, const Monitor&, int, double2*, cudaStream_t);
template int mpa_levels<double>(const Split&, int, int, int, double2*, double2*, double2*, double2*, const NodeC*,
                                const int*, const double*, const Monitor&, int, double2*, cudaStream_t);

}  // namespace host
}  // namespace mpa

namespace mpa {
namespace host {

Monitor monitor(const mpa_plan* p) {
    Monitor m{};
    m.err = reinterpret_cast<unsigned int*>(p->ws + p->off_err);
    m.conv = reinterpret_cast<ConvState*>(p->ws + p->off_conv);
    m.dprev = reinterpret_cast<float2*>(p->ws + p->off_dprev);
    m.spin_limit = kSpinLimit;
    const size_t hi = p->dbg_hi ? p->dbg_hi : p->ws_bytes;
    m.dbg = DbgRange{reinterpret_cast<const char*>(p->ws + p->dbg_lo), reinterpret_cast<const char*>(p->ws + hi), m.err};
    return m;
}

int interval_type(const mpa_plan* p, double z0, int* t) {
    if (p->n_types == 1) {
        *t = 0;
        return MPA_OK;
    }
    const double u = z0 - std::floor(z0 / p->map.period + 1e-12) * p->map.period;
    double r;
    if (!whole(u / p->L, &r)) return MPA_ERR_GRID;
    long q = (long)r % p->n_types;
    if (q < 0) q += p->n_types;
    *t = (int)q;
    return MPA_OK;
}

template <typename T>
int run_interval(mpa_plan* p, int type, long n_amp, int scan_mode, double2* out, cudaStream_t st) {
    const int* toff = reinterpret_cast<const int*>(p->ws + p->off_toff);
    const double* gains = reinterpret_cast<const double*>(p->ws + p->off_gains);
    if (n_amp < 0 || n_amp >= kMaxAmpsPerInterval) return MPA_ERR_GRID;
    return mpa_levels<T>(p->sp, p->M, p->n_iter, 1, reinterpret_cast<cx<T>*>(p->ws + p->off_psi),
                         p->has_work ? reinterpret_cast<cx<T>*>(p->ws + p->off_work2) : nullptr,
                         reinterpret_cast<cx<T>*>(p->ws + p->off_psi0c),
                         reinterpret_cast<double2*>(p->ws + p->off_state),
                         reinterpret_cast<const NodeC*>(p->ws + p->off_nodes), toff + type, gains + n_amp,
                         monitor(p), scan_mode, out, st);
}
template int run_interval<float>(mpa_plan*, int, long, int, double2*, cudaStream_t);
template int run_interval<double>(mpa_plan*, int, long, int, double2*, cudaStream_t);

}  // namespace host
}  // namespace mpa

namespace {

// Wavefront schedule of one interval (FP32): node blocks of B move through
// the n_iter levels one step at a time; at step s level n works on block
// s - n.  Each step is one row pass per active block and one wavefront
// column pass for all active blocks.  Results equal the level-synchronous
// schedule up to the summation order of the FP32 sums.
int run_interval_wf(mpa_plan* p, int type, double gain, double2* out, cudaStream_t st) {
    const Split& s = p->sp;
    const long long N = s.N;
    const int M = p->M, S = p->n_iter, B = p->B;
    const int nb = (M + B - 1) / B;
    float2* work = reinterpret_cast<float2*>(p->ws + p->off_work);
    float2* y0 = reinterpret_cast<float2*>(p->ws + p->off_y0);
    float2* psi0c = reinterpret_cast<float2*>(p->ws + p->off_psi0c);
    double2* state = reinterpret_cast<double2*>(p->ws + p->off_state);
    const NodeC* nodes = reinterpret_cast<const NodeC*>(p->ws + p->off_nodes) + (size_t)type * (M + 1);
    unsigned int* err = reinterpret_cast<unsigned int*>(p->ws + p->off_err);
    const long long slot_stride = (long long)B * N;
    auto nn = [&](int b) { return (b < nb) ? ((b + 1) * B <= M ? B : M - b * B) : 0; };
    auto kc = [&](int mode, const float2* src, long long src_stride, float2* dst, int first, int count) {
        KCParams<float> c{};
        c.src = src;
        c.src_stride = src_stride;
        c.dst = dst;
        c.dst_stride = N;
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.ncols = (long long)count * s.N1;
        c.npl = count;
        c.nodes = nodes + first;
        c.loff = reinterpret_cast<const int*>(p->ws + p->off_toff);  // entry 0 is offset 0
        return kc_launch<float>(mode, s.logN2, c, st);
    };
    auto kr = [&](float2* data, int count) {
        KRParams<float> r{data, (long long)count * s.N2, N, s.logN, (int)s.N2, (float)(1.0 / (double)N), 0.f};
        return kr_launch<float>(KR_MPA, s.logN1, r, st);
    };
    // node 0: V_0 (the same for every iteration)
    MPA_TRY(kc(KC_MPA_PRE, psi0c, 0, y0, 0, 1));
    MPA_TRY(kr(y0, 1));
    MPA_TRY(kc(KC_MPA_POST, y0, N, y0, 0, 1));
    // first iteration inputs of the first S blocks
    for (int b = 0; b < S && b < nb; ++b) MPA_TRY(kc(KC_MPA_PRE, psi0c, 0, work + (long long)(b % S) * slot_stride, 1 + b * B, nn(b)));
    KCWParams w{};
    w.work = work;
    w.slot_stride = slot_stride;
    w.N = N;
    w.logN = s.logN;
    w.N1 = (int)s.N1;
    w.logN1 = s.logN1;
    w.M = M;
    w.nodes = nodes;
    w.psi0 = psi0c;
    w.v0 = y0;
    w.Rg = reinterpret_cast<float2*>(p->ws + p->off_R);
    w.Cg = reinterpret_cast<float2*>(p->ws + p->off_C);
    w.D = reinterpret_cast<double2*>(p->ws + p->off_D);
    for (int step = 0; step < nb + S - 1; ++step) {
        w.n_jobs = 0;
        for (int n = 0; n < S; ++n) {
            const int b = step - n;
            if (b < 0 || b >= nb) continue;
            KCWJob& j = w.job[w.n_jobs++];
            j.level = n;
            j.slot = b % S;
            j.node_first = 1 + b * B;
            j.n_nodes = nn(b);
            j.last = (n == S - 1);
            j.head_first = 1 + (b + S) * B;
            j.n_head = j.last ? nn(b + S) : 0;
        }
        // row passes (steps 3-4): one launch over all slots when every slot is
        // busy (the slots are contiguous), else one per active block
        if (w.n_jobs == S) {
            MPA_TRY(kr(work, S * B));
        } else {
            for (int i = 0; i < w.n_jobs; ++i)
                MPA_TRY(kr(work + (long long)w.job[i].slot * slot_stride, w.job[i].n_nodes));
        }
        MPA_TRY(kcw_launch(s.logN2, w, st));
    }
    // step 7 (or psi_M only)
    const NodeC nodeM = p->nodes[(size_t)type * (M + 1) + M];
    MPA_TRY(reconstruct_launch(state, psi0c, w.D, nodeM, gain, N, err, out, st));
    return MPA_OK;
}

template <typename T>
int propagate_t(mpa_plan* p, void* field, double z_from, double z_to, cudaStream_t st) {
    const Split& s = p->sp;
    const double L = p->L;
    double qf, ni;
    if (!(z_from >= -1e-12) || !(z_to >= z_from) || z_to > p->map.length * (1 + 1e-12) + 1e-9) return MPA_ERR_GRID;
    if (!whole(z_from / L, &qf) || !whole((z_to - z_from) / L, &ni) || ni > kMaxIntervals) return MPA_ERR_GRID;
    const long n_int = (long)ni;
    std::vector<int> types((size_t)n_int);
    std::vector<long> amps((size_t)n_int);
    for (long q = 0; q < n_int; ++q) {
        const double z0 = z_from + L * (double)q;
        if (p->map.amp_inside(z0, z0 + L)) return MPA_ERR_GRID;
        int t;
        if (interval_type(p, z0, &t) != MPA_OK) return MPA_ERR_GRID;
        types[(size_t)q] = t;
        amps[(size_t)q] = p->map.amps(z0, z0 + L);
    }
    cx<T>* f = reinterpret_cast<cx<T>*>(field);
    cx<T>* psi = reinterpret_cast<cx<T>*>(p->ws + p->off_psi);
    double2* state = reinterpret_cast<double2*>(p->ws + p->off_state);
    cx<T>* psi0c = reinterpret_cast<cx<T>*>(p->ws + p->off_psi0c);
    // A_hat(z_from) = F[A] -> FP64 state and its working copy
    int rc = fft_forward<T>(s, f, psi, st);
    if (rc) return rc;
    MPA_TRY(to_state_launch<T>(psi, state, sizeof(T) == 4 ? psi0c : nullptr, s.N, st));
    for (long q = 0; q < n_int; ++q) {
        NvtxRange nvq("interval");
        rc = p->wf ? run_interval_wf(p, types[(size_t)q], std::exp((double)amps[(size_t)q] * p->map.z_a * p->map.gamma),
                                     nullptr, st)
                   : run_interval<T>(p, types[(size_t)q], amps[(size_t)q], 1, nullptr, st);
        if (rc) return rc;
    }
    // A(z_to) = F^-1[A_hat]
    MPA_TRY(from_state_launch<T>(state, psi, s.N, st));
    return fft_inverse<T>(s, psi, f, st);
}

template <typename T>
int interval_t(mpa_plan* p, const void* psi0, void* psiM, double z0, cudaStream_t st) {
    double q;
    if (!whole(z0 / p->L, &q) || z0 < -1e-12 || z0 + p->L > p->map.length * (1 + 1e-12) + 1e-9) return MPA_ERR_GRID;
    if (p->map.amp_inside(z0, z0 + p->L)) return MPA_ERR_GRID;
    int t;
    if (interval_type(p, z0, &t) != MPA_OK) return MPA_ERR_GRID;
    double2* state = reinterpret_cast<double2*>(p->ws + p->off_state);
    cx<T>* psi0c = reinterpret_cast<cx<T>*>(p->ws + p->off_psi0c);
    MPA_TRY(cudaMemcpyAsync(state, psi0, (size_t)p->sp.N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    if (sizeof(T) == 4) MPA_TRY(from_state_launch<T>(state, psi0c, p->sp.N, st));
    if (p->wf) return run_interval_wf(p, t, 1.0, reinterpret_cast<double2*>(psiM), st);
    return run_interval<T>(p, t, 0, 2, reinterpret_cast<double2*>(psiM), st);
}

template <typename T>
int ss_t(const HostMap& m, const Split& s, double T_ps, double dz, void* field, double z_from, double z_to,
         void* ws, cudaStream_t st) {
    double kk;
    if (!(z_from >= -1e-12) || !(z_to > z_from) || z_to > m.length * (1 + 1e-12) + 1e-9) return MPA_ERR_GRID;
    if (!whole((z_to - z_from) / dz, &kk) || kk < 1 || kk > kMaxIntervals) return MPA_ERR_GRID;
    const long K = (long)kk;
    cx<T>* f = reinterpret_cast<cx<T>*>(field);
    cx<T>* w = reinterpret_cast<cx<T>*>(ws);
    auto flow = [&](double za, double zb) {
        NodeC c{};
        phase_consts(m.integ(za, zb, 1), m.integ(za, zb, 2), T_ps, &c);
        c.pre = std::exp(m.G(za, zb) + (double)m.amps(za, zb) * m.z_a * m.gamma);
        c.post = 1.0;
        return c;
    };
    // time data -> (transpose) -> forward row pass; the column pass of every
    // step finishes the forward transform, applies the linear step and starts
    // the inverse transform.
    MPA_TRY(transpose_launch<T>(f, w, s.N1, s.N2, st));
    KRParams<T> r{w, s.N2, s.N, s.logN, (int)s.N2, (T)(1.0 / (double)s.N), T(0)};
    MPA_TRY(kr_launch<T>(KR_FWD, s.logN1, r, st));
    KCParams<T> c{};
    c.src = w;
    c.dst = w;
    c.N = s.N;
    c.logN = s.logN;
    c.N1 = (int)s.N1;
    c.logN1 = s.logN1;
    c.ncols = s.N1;
    c.flow = flow(z_from, z_from + 0.5 * dz);
    MPA_TRY(kc_launch<T>(KC_SS_STEP, s.logN2, c, st));
    for (long k = 0; k < K; ++k) {
        const double zk = z_from + dz * (double)k;
        r.rot = (T)m.integ(zk, zk + dz, 3);
        MPA_TRY(kr_launch<T>(KR_SS, s.logN1, r, st));
        const double za = zk + 0.5 * dz;
        const double zb = (k == K - 1) ? z_to : za + dz;
        c.flow = flow(za, zb);
        MPA_TRY(kc_launch<T>(KC_SS_STEP, s.logN2, c, st));
    }
    KRParams<T> ri{w, s.N2, s.N, s.logN, (int)s.N2, (T)(1.0 / (double)s.N), T(0)};
    MPA_TRY(kr_launch<T>(KR_INV, s.logN1, ri, st));
    MPA_TRY(transpose_launch<T>(w, f, s.N2, s.N1, st));
    return MPA_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

int mpa_plan_create(const mpa_fiber_map* map, const mpa_plan_params* prm, mpa_plan** out) {
    return abi_call([&]() -> int {
        if (!map || !prm || !out) return MPA_ERR_INVALID_ARG;
        *out = nullptr;
        if (prm->precision != MPA_FP32 && prm->precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
        if (!(prm->T_ps > 0.0) || !(prm->L_km > 0.0) || prm->M < 1 || prm->M > kMaxNodes || prm->n_iter < 1)
            return MPA_ERR_INVALID_ARG;
        if (prm->schedule < MPA_SCHEDULE_AUTO || prm->schedule > MPA_SCHEDULE_WAVEFRONT) return MPA_ERR_INVALID_ARG;
        std::unique_ptr<mpa_plan> p(new mpa_plan());  // released to *out on success
        int rc = p->map.init(map);
        if (rc == MPA_OK) rc = split_n(prm->N, prm->precision, &p->sp);
        if (rc != MPA_OK) return rc;
        // FP32 plans whose spectra fit one CTA use the on-chip node transform by
        // default (1.75x the three passes on the 2^14-mode link); the cluster
        // form (2^15, 2^16) and FP64 plans are chosen by set_split(0) or tuning
        p->sp.onchip = prm->precision == MPA_FP32 && prm->schedule != MPA_SCHEDULE_WAVEFRONT &&
                       onchip_ok(prm->N, MPA_FP32) && prm->N <= (1ll << 14);
        p->T = prm->T_ps;
        p->L = prm->L_km;
        p->M = prm->M;
        p->n_iter = prm->n_iter;
        p->prec = prm->precision;
        double r;
        if (whole(p->map.period / p->L, &r) && r >= 1) {
            if (r > kMaxIntervalTypes) return MPA_ERR_GRID;
            p->n_types = (int)r;
        } else if (whole(p->L / p->map.period, &r) && r >= 1) {
            p->n_types = 1;
        } else {
            return MPA_ERR_GRID;
        }
        // per-node constants of Eq. (6) for each interval start u0 = t L in the period
        const int M = p->M;
        const double dz = p->L / M;
        p->nodes.resize((size_t)p->n_types * (M + 1));
        for (int t = 0; t < p->n_types; ++t) {
            const double u0 = p->L * t;
            for (int j = 0; j <= M; ++j) {
                const double zr = (j == M) ? p->L : dz * j;
                NodeC& c = p->nodes[(size_t)t * (M + 1) + j];
                phase_consts(p->map.integ(u0, u0 + zr, 1), p->map.integ(u0, u0 + zr, 2), p->T, &c);
                c.pre = std::exp(p->map.G(u0, u0 + zr));
                double sig;
                if (j == 0) sig = p->map.side(u0, 3, +1);
                else if (j == M) sig = p->map.side(u0 + zr, 3, -1);
                else sig = 0.5 * (p->map.side(u0 + zr, 3, -1) + p->map.side(u0 + zr, 3, +1));
                c.post = sig * dz / c.pre;
            }
        }
        p->csize = p->prec == MPA_FP32 ? sizeof(float2) : sizeof(double2);
        const size_t N = (size_t)p->sp.N;
        // schedule: the wavefront needs FP32 and whole column tiles per node
        // (column length >= 128 keeps its shared memory within the 227 KB limit)
        p->wf = prm->schedule == MPA_SCHEDULE_WAVEFRONT && p->prec == MPA_FP32 && p->n_iter <= 8 && p->sp.logN2 >= 7 &&
                p->sp.N1 >= kcw_tile_cols(p->sp.logN2) && p->sp.N1 % kcw_tile_cols(p->sp.logN2) == 0;
        if (prm->schedule == MPA_SCHEDULE_WAVEFRONT && !p->wf) return MPA_ERR_INVALID_ARG;
        if (p->wf) {
            // B nodes per block: about 256 MiB of node buffers over the n_iter slots
            const size_t per = (size_t)p->n_iter * N * sizeof(float2);
            long b = (long)((256ull << 20) / per);
            b = b < 1 ? 1 : b > 16 ? 16 : b;
            p->B = (int)(b < M ? b : M);
            const size_t S = (size_t)p->n_iter;
            p->off_work = 0;
            p->off_y0 = align256(p->off_work + S * (size_t)p->B * N * sizeof(float2));
            p->off_R = align256(p->off_y0 + N * sizeof(float2));
            p->off_C = align256(p->off_R + S * N * sizeof(float2));
            p->off_D = align256(p->off_C + S * N * sizeof(float2));
            p->off_state = align256(p->off_D + N * sizeof(double2));
            p->off_psi0c = align256(p->off_state + N * sizeof(double2));
            p->off_psi = p->off_work;  // scratch of the entry/exit transforms
            p->off_nodes = align256(p->off_psi0c + N * sizeof(float2));
            p->off_toff = align256(p->off_nodes + p->nodes.size() * sizeof(NodeC));
            p->off_gains = align256(p->off_toff + (size_t)p->n_types * sizeof(int));
            p->off_err = align256(p->off_gains + kMaxAmpsPerInterval * sizeof(double));
            p->off_conv = align256(p->off_err + sizeof(unsigned int));
            p->off_dprev = align256(p->off_conv + sizeof(ConvState));
            p->ws_need = align256(p->off_dprev);  // the wavefront schedule has no increment check
            *out = p.release();
            return MPA_OK;
        }
        p->off_psi = 0;
        p->has_work = wants_work_buffers(p->sp.N, p->prec);
        p->off_work2 = align256(p->off_psi + (size_t)(M + 1) * N * p->csize);
        p->off_state = p->has_work ? align256(p->off_work2 + (size_t)(M + 1) * N * p->csize) : p->off_work2;
        p->off_psi0c = align256(p->off_state + N * sizeof(double2));
        const size_t psi0c_bytes = p->prec == MPA_FP32 ? N * sizeof(float2) : 0;
        if (p->prec == MPA_FP64) p->off_psi0c = p->off_state;  // the FP64 state is its own working copy
        const size_t after_psi0c =
            p->prec == MPA_FP32 ? p->off_psi0c + psi0c_bytes : p->off_state + N * sizeof(double2);
        p->off_nodes = align256(after_psi0c);
        p->off_toff = align256(p->off_nodes + p->nodes.size() * sizeof(NodeC));
        p->off_gains = align256(p->off_toff + (size_t)p->n_types * sizeof(int));
        p->off_err = align256(p->off_gains + kMaxAmpsPerInterval * sizeof(double));
        p->off_conv = align256(p->off_err + sizeof(unsigned int));
        p->off_dprev = align256(p->off_conv + sizeof(ConvState));
        p->ws_need = align256(p->off_dprev + (p->n_iter > 1 ? N * sizeof(float2) : 0));
        *out = p.release();
        return MPA_OK;
    });
}

int mpa_plan_workspace_size(const mpa_plan* p, size_t* bytes) {
    if (!p || !bytes) return MPA_ERR_INVALID_ARG;
    *bytes = p->ws_need;
    return MPA_OK;
}

int mpa_plan_set_workspace(mpa_plan* p, void* ws, size_t bytes) {
    return abi_call([&]() -> int {
        if (!p || !ws) return MPA_ERR_INVALID_ARG;
        if (bytes < p->ws_need || ((uintptr_t)ws & 255u) != 0) return MPA_ERR_WORKSPACE;
        p->ws = reinterpret_cast<unsigned char*>(ws);
        p->ws_bytes = bytes;
        MPA_TRY(cudaMemcpy(p->ws + p->off_nodes, p->nodes.data(), p->nodes.size() * sizeof(NodeC),
                           cudaMemcpyHostToDevice));
        std::vector<int> toff((size_t)p->n_types);
        for (int t = 0; t < p->n_types; ++t) toff[(size_t)t] = t * (p->M + 1);
        MPA_TRY(cudaMemcpy(p->ws + p->off_toff, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice));
        double gains[kMaxAmpsPerInterval];
        for (int a = 0; a < kMaxAmpsPerInterval; ++a) gains[a] = std::exp((double)a * p->map.z_a * p->map.gamma);
        MPA_TRY(cudaMemcpy(p->ws + p->off_gains, gains, sizeof(gains), cudaMemcpyHostToDevice));
        MPA_TRY(cudaMemset(p->ws + p->off_err, 0, sizeof(unsigned int)));
        MPA_TRY(cudaMemset(p->ws + p->off_conv, 0, sizeof(ConvState)));
        return MPA_OK;
    });
}

}  // extern "C"

namespace {

// The split with column length 2^l if every pass (and the reverse-mode
// tiling, one node per tile, for N >= 2^13) supports it.
bool admissible_split(const mpa_plan* p, int l, Split* s) {
    if (split_with(p->sp.N, p->prec, l, s) != MPA_OK) return false;
    if (s->logN >= 13) {
        const bool f32 = p->prec == MPA_FP32;
        const int gc = f32 ? kca_tile_cols<float>(s->logN2) : kca_tile_cols<double>(s->logN2);
        const int gr = f32 ? kra_tile_rows<float>(s->logN1) : kra_tile_rows<double>(s->logN1);
        if (gc <= 0 || gr <= 0 || gc > s->N1 || gr > s->N2) return false;
    }
    return true;
}

}  // namespace

extern "C" {

int mpa_plan_set_split(mpa_plan* p, int32_t log2_n2) {
    if (!p) return MPA_ERR_INVALID_ARG;
    if (p->wf) return log2_n2 == p->sp.logN2 ? MPA_OK : MPA_ERR_UNSUPPORTED_N;
    if (log2_n2 == 0) {
        // on-chip node transforms; the entry/exit transforms keep a four-step split
        if (!onchip_ok(p->sp.N, p->prec)) return MPA_ERR_UNSUPPORTED_N;
        if (p->sp.onchip) return MPA_OK;
        Split s;
        if (split_n(p->sp.N, p->prec, &s) != MPA_OK) return MPA_ERR_UNSUPPORTED_N;
        s.onchip = true;
        p->sp = s;
        return MPA_OK;
    }
    Split s;
    if (!admissible_split(p, log2_n2, &s)) return MPA_ERR_UNSUPPORTED_N;
    p->sp = s;
    return MPA_OK;
}

int mpa_plan_autotune(mpa_plan* p, mpa_stream stream, int32_t* log2_n2) {
    NvtxRange nv("mpa_plan_autotune");
    if (!p) return MPA_ERR_INVALID_ARG;
    if (!p->ws) return MPA_ERR_WORKSPACE;
    if (log2_n2) *log2_n2 = p->sp.onchip ? 0 : p->sp.logN2;
    if (p->wf) return MPA_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const Split keep = p->sp;
    const size_t N = (size_t)keep.N;
    const bool f32 = p->prec == MPA_FP32;
    cudaEvent_t e0, e1;
    MPA_TRY(cudaEventCreate(&e0));
    MPA_TRY(cudaEventCreate(&e1));
    Split best = keep;
    float best_ms = -1.f;
    int rc = MPA_OK;
    // candidates: the on-chip node transform (reported as column length 2^0)
    // where N fits, then every admissible four-step split
    for (int l = keep.logN / 2 - 4; l <= keep.logN / 2 + 3 && rc == MPA_OK; ++l) {
        Split s;
        if (l == keep.logN / 2 - 4) {
            if (!onchip_ok(keep.N, p->prec) || split_n(keep.N, p->prec, &s) != MPA_OK) continue;
            s.onchip = true;
        } else if (!admissible_split(p, l, &s)) {
            continue;
        }
        p->sp = s;
        // a zero field: the timing does not depend on the values
        if (cudaMemsetAsync(p->ws + p->off_state, 0, N * sizeof(double2), st) != cudaSuccess ||
            (f32 && cudaMemsetAsync(p->ws + p->off_psi0c, 0, N * sizeof(float2), st) != cudaSuccess)) {
            rc = cuda_fail(cudaGetLastError());
            break;
        }
        float ms = 0.f;
        for (int rep = 0; rep < 2 && rc == MPA_OK; ++rep) {  // rep 0 warms up (first launches, attributes)
            if (cudaEventRecord(e0, st) != cudaSuccess) { rc = MPA_ERR_CUDA; break; }
            rc = f32 ? run_interval<float>(p, 0, 0, 1, nullptr, st) : run_interval<double>(p, 0, 0, 1, nullptr, st);
            if (rc == MPA_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = cuda_fail(cudaGetLastError());
        }
        if (rc == MPA_OK && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->sp = best;
    if (rc != MPA_OK) p->sp = keep;
    if (log2_n2) *log2_n2 = p->sp.onchip ? 0 : p->sp.logN2;
    MPA_TRY(cudaMemsetAsync(p->ws + p->off_err, 0, sizeof(unsigned int), st));
    MPA_TRY(cudaMemsetAsync(p->ws + p->off_conv, 0, sizeof(ConvState), st));
    return rc;
}

int mpa_propagate(mpa_plan* p, void* field, double z_from_km, double z_to_km, mpa_stream stream) {
    return abi_call([&]() -> int {
        EntryRange nv("mpa_propagate", stream);
        if (!p || !field) return MPA_ERR_INVALID_ARG;
        if (!p->ws) return MPA_ERR_WORKSPACE;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        return p->prec == MPA_FP32 ? propagate_t<float>(p, field, z_from_km, z_to_km, st)
                                   : propagate_t<double>(p, field, z_from_km, z_to_km, st);
    });
}

int mpa_interval(mpa_plan* p, const void* psi0, void* psiM, double z0_km, mpa_stream stream) {
    EntryRange nv("mpa_interval", stream);
    if (!p || !psi0 || !psiM) return MPA_ERR_INVALID_ARG;
    if (!p->ws) return MPA_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return p->prec == MPA_FP32 ? interval_t<float>(p, psi0, psiM, z0_km, st)
                               : interval_t<double>(p, psi0, psiM, z0_km, st);
}

int mpa_plan_status(mpa_plan* p, mpa_stream stream) {
    if (!p) return MPA_ERR_INVALID_ARG;
    if (!p->ws) return MPA_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned int h = 0;
    MPA_TRY(cudaMemcpyAsync(&h, p->ws + p->off_err, sizeof(h), cudaMemcpyDeviceToHost, st));
    MPA_TRY(cudaStreamSynchronize(st));
    MPA_TRY(cudaMemsetAsync(p->ws + p->off_err, 0, sizeof(unsigned int), st));
    return status_of_error_word(h);
}

int mpa_plan_contraction(mpa_plan* p, mpa_stream stream, double* worst) {
    if (!p || !worst) return MPA_ERR_INVALID_ARG;
    if (!p->ws) return MPA_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ConvState c{};
    MPA_TRY(cudaMemcpyAsync(&c, p->ws + p->off_conv, sizeof(c), cudaMemcpyDeviceToHost, st));
    MPA_TRY(cudaStreamSynchronize(st));
    *worst = c.worst;
    const double zero = 0.0;
    MPA_TRY(cudaMemcpyAsync(p->ws + p->off_conv + offsetof(ConvState, worst), &zero, sizeof(double),
                            cudaMemcpyHostToDevice, st));
    MPA_TRY(cudaStreamSynchronize(st));
    return MPA_OK;
}

int mpa_plan_check_scales(const mpa_plan* p, double peak_power_W, double pulse_width_ps, double* z_nl_km,
                          double* z_disp_km, int32_t* flags) {
    if (!p || !(peak_power_W > 0.0) || !(pulse_width_ps > 0.0) || !std::isfinite(peak_power_W) ||
        !std::isfinite(pulse_width_ps))
        return MPA_ERR_INVALID_ARG;
    // typical sigma and |beta2| of the map: the largest sigma (the strongest
    // nonlinearity) and the length-weighted mean |beta2| over a period
    double smax = 0.0, b2 = 0.0;
    for (const auto& s : p->map.seg) {
        smax = std::fmax(smax, std::fabs(s.sigma_per_W_km));
        b2 += std::fabs(s.beta2_ps2_per_km) * s.length_km;
    }
    b2 /= p->map.period;
    const double znl = smax > 0.0 ? 1.0 / (smax * peak_power_W) : HUGE_VAL;
    const double zd = b2 > 0.0 ? pulse_width_ps * pulse_width_ps / b2 : HUGE_VAL;
    int32_t f = 0;
    if (!(znl > zd)) f |= MPA_SCALE_STRONG_NONLINEARITY;
    if (!(p->L < znl)) f |= MPA_SCALE_L_ABOVE_ZNL;
    if (p->L > zd) f |= MPA_SCALE_L_ABOVE_ZDISP;
    if (z_nl_km) *z_nl_km = znl;
    if (z_disp_km) *z_disp_km = zd;
    if (flags) *flags = f;
    return (f & (MPA_SCALE_STRONG_NONLINEARITY | MPA_SCALE_L_ABOVE_ZNL)) ? MPA_ERR_SCALES : MPA_OK;
}

void mpa_plan_destroy(mpa_plan* p) { delete p; }

int ss_workspace_size(int64_t N, int32_t precision, size_t* bytes) {
    if (!bytes || (precision != MPA_FP32 && precision != MPA_FP64)) return MPA_ERR_INVALID_ARG;
    Split s;
    int rc = split_n(N, precision, &s);
    if (rc) return rc;
    *bytes = align256((size_t)N * (precision == MPA_FP32 ? sizeof(float2) : sizeof(double2)));
    return MPA_OK;
}

int ss_propagate(const mpa_fiber_map* map, int64_t N, double T_ps, double dz_km, int32_t precision, void* field,
                 double z_from_km, double z_to_km, void* workspace, size_t ws_bytes, mpa_stream stream) {
    return abi_call([&]() -> int {
        EntryRange nv("ss_propagate", stream);
        if (!map || !field || !workspace || !(T_ps > 0.0) || !(dz_km > 0.0)) return MPA_ERR_INVALID_ARG;
        if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
        HostMap m;
        int rc = m.init(map);
        if (rc) return rc;
        Split s;
        rc = split_n(N, precision, &s);
        if (rc) return rc;
        size_t need = 0;
        ss_workspace_size(N, precision, &need);
        if (ws_bytes < need) return MPA_ERR_WORKSPACE;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        return precision == MPA_FP32 ? ss_t<float>(m, s, T_ps, dz_km, field, z_from_km, z_to_km, workspace, st)
                                     : ss_t<double>(m, s, T_ps, dz_km, field, z_from_km, z_to_km, workspace, st);
    });
}

int mpa_fft(int64_t N, int32_t precision, int32_t sign, void* data, void* workspace, size_t ws_bytes,
            mpa_stream stream) {
    EntryRange nv("mpa_fft", stream);
    if (!data || !workspace || (sign != 1 && sign != -1)) return MPA_ERR_INVALID_ARG;
    if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
    Split s;
    int rc = split_n(N, precision, &s);
    if (rc) return rc;
    size_t need = 0;
    ss_workspace_size(N, precision, &need);
    if (ws_bytes < need) return MPA_ERR_WORKSPACE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)N * (precision == MPA_FP32 ? sizeof(float2) : sizeof(double2));
    if (precision == MPA_FP32) {
        float2* d = reinterpret_cast<float2*>(data);
        float2* w = reinterpret_cast<float2*>(workspace);
        rc = sign > 0 ? fft_forward<float>(s, d, w, st) : fft_inverse<float>(s, d, w, st);
    } else {
        double2* d = reinterpret_cast<double2*>(data);
        double2* w = reinterpret_cast<double2*>(workspace);
        rc = sign > 0 ? fft_forward<double>(s, d, w, st) : fft_inverse<double>(s, d, w, st);
    }
    if (rc) return rc;
    MPA_TRY(cudaMemcpyAsync(data, workspace, bytes, cudaMemcpyDeviceToDevice, st));
    return MPA_OK;
}

double mpa_gamma_from_db_per_km(double db_per_km) { return db_per_km * std::log(10.0) / 20.0; }

const char* mpa_status_string(int status) {
    switch (status) {
        case MPA_OK: return "ok";
        case MPA_ERR_INVALID_ARG: return "invalid argument";
        case MPA_ERR_UNSUPPORTED_N: return "unsupported N (power of two in [2^8, 2^25], 2^24 for FP64)";
        case MPA_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case MPA_ERR_CUDA: return "CUDA error";
        case MPA_ERR_GRID: return "z-grid inconsistent with the fiber map";
        case MPA_ERR_NONFINITE: return "non-finite value produced";
        case MPA_ERR_DIVERGED: return "Picard iteration diverged (the increment grew between iterations)";
        case MPA_ERR_SCALES: return "scales outside the weak-nonlinearity regime of the method";
        case MPA_ERR_TIMEOUT: return "a bounded wait of a persistent kernel ran out (results incomplete)";
        case MPA_ERR_BOUNDS: return "debug build: an access outside the checked buffer range was skipped";
        case MPA_ERR_HOST_MEMORY: return "host memory allocation failed";
    }
    return "unknown status";
}

const char* mpa_last_cuda_error(void) { return mpa::host::g_cuda_err.c_str(); }

int64_t mpa_kernel_launches(void) { return (int64_t)g_launches.load(); }

void mpa_profile(int enable) {
    if (enable) {
        prof_reset();
        call_timing_reset();
    }
    g_prof_on.store(enable != 0);
}

int mpa_profile_read(int kind, double* total_ms, int64_t* launches, double* bytes) {
    if (kind < 0 || kind >= PK_COUNT || !total_ms || !launches || !bytes) return MPA_ERR_INVALID_ARG;
    long long n = 0;
    cudaError_t e = prof_read(kind, total_ms, &n, bytes);
    *launches = n;
    if (e != cudaSuccess) return cuda_fail(e);
    return MPA_OK;
}

int32_t mpa_debug_bounds_checked(void) { return MPA_DEBUG_BOUNDS ? 1 : 0; }

int mpa_debug_set_bounds(mpa_plan* p, size_t lo, size_t hi) {
    if (!p || lo > hi) return MPA_ERR_INVALID_ARG;
    if (!p->ws) return MPA_ERR_WORKSPACE;
    if (hi > p->ws_bytes) return MPA_ERR_INVALID_ARG;
    p->dbg_lo = lo;
    p->dbg_hi = hi;  // 0 (with lo 0): the whole workspace
    return MPA_OK;
}

int mpa_last_timing(double* ms, const char** entry) {
    if (!ms) return MPA_ERR_INVALID_ARG;
    bool have = false;
    const cudaError_t e = call_timing_read(ms, entry, &have);
    if (e != cudaSuccess) return cuda_fail(e);
    return have ? MPA_OK : MPA_ERR_INVALID_ARG;
}

const char* mpa_profile_kind_name(int kind) {
    static const char* names[PK_COUNT] = {"kc_mpa_pre", "kc_mpa_post", "kc_ss_step", "kc_fft", "kr_mpa",
                                          "kr_ss", "kr_fft", "scan", "aux", "kc_wavefront",
                                          "kc_adjoint", "kr_adjoint", "adjoint_aux", "kn_mpa"};
    return (kind >= 0 && kind < PK_COUNT) ? names[kind] : nullptr;
}

}  // extern "C"
