// Reverse mode of mpa_propagate: gradients of a real loss with respect to the
// input field and to sigma and beta2 of every physical segment.
//
// Schedule: a forward pass stores A_hat at every interval start (FP64
// checkpoints).  The intervals are then walked backwards.  For each one the
// levels of MPA steps 2-5 are recomputed from its checkpoint with every
// level kept (psi^{(n)}, A^{(n)}(t) and V^{(n)} at all nodes), and the
// levels are reversed one by one (adjoint.cuh): reverse scan, then the two
// column passes and the row pass of the node transforms.  Per-node partial
// sums of the parameter gradients go to a small device table that the host
// folds into the segments at the end.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "adj_launch.h"
#include "plan.h"

using namespace mpa;
using namespace mpa::host;

namespace {

struct AdjLayout {
    long n_int = 0;
    double z_from = 0.0;
    int acc_stride = 0;   // per interval: M+1 beta2 sums, M+1 sigma sums, the step-7 beta2 sum
    long long tiles = 0;  // largest number of partial sums of one launch
    size_t off_ck = 0, off_psi = 0, off_a = 0, off_v = 0, off_g = 0, off_gx = 0, off_gs = 0, off_p0 = 0, off_part = 0,
           off_acc = 0, off_adjc = 0, need = 0;
    std::vector<int> types;
    std::vector<long> amps;
};

int n_periods_of(const HostMap& m) { return (int)std::lround(m.length / m.period); }

int adj_layout(const mpa_plan* p, double z_from, double z_to, AdjLayout* a) {
    if (p->wf) return MPA_ERR_INVALID_ARG;
    if (p->sp.logN < 13) return MPA_ERR_UNSUPPORTED_N;
    const double L = p->L;
    double qf, ni;
    if (!(z_from >= -1e-12) || !(z_to > z_from) || z_to > p->map.length * (1 + 1e-12) + 1e-9) return MPA_ERR_GRID;
    if (!whole(z_from / L, &qf) || !whole((z_to - z_from) / L, &ni) || ni < 1 || ni > kMaxIntervals)
        return MPA_ERR_GRID;
    a->n_int = (long)ni;
    a->z_from = z_from;
    a->types.assign((size_t)a->n_int, 0);
    a->amps.assign((size_t)a->n_int, 0);
    for (long q = 0; q < a->n_int; ++q) {
        const double z0 = z_from + L * (double)q;
        if (p->map.amp_inside(z0, z0 + L)) return MPA_ERR_GRID;
        int t;
        if (interval_type(p, z0, &t) != MPA_OK) return MPA_ERR_GRID;
        a->types[(size_t)q] = t;
        a->amps[(size_t)q] = p->map.amps(z0, z0 + L);
        if (a->amps[(size_t)q] >= kMaxAmpsPerInterval) return MPA_ERR_GRID;
    }
    const Split& s = p->sp;
    const size_t N = (size_t)s.N, cs = p->csize, nodes = (size_t)p->M + 1, S = (size_t)p->n_iter;
    const bool f32 = p->prec == MPA_FP32;
    const int gc = f32 ? kca_tile_cols<float>(s.logN2) : kca_tile_cols<double>(s.logN2);
    const int gr = f32 ? kra_tile_rows<float>(s.logN1) : kra_tile_rows<double>(s.logN1);
    // every column tile inside one node's N1 columns, every row tile inside its N2 rows
    if (gc <= 0 || gr <= 0 || gc > s.N1 || gr > s.N2) return MPA_ERR_UNSUPPORTED_N;
    long long t = (long long)nodes * (s.N1 / gc);
    t = std::max(t, (long long)nodes * (s.N2 / gr));
    t = std::max(t, (long long)((N + 255) / 256));
    a->tiles = t;
    a->acc_stride = 2 * (int)nodes + 1;
    a->off_ck = 0;
    a->off_psi = align256(a->off_ck + (size_t)(a->n_int + 1) * N * sizeof(double2));
    a->off_a = align256(a->off_psi + (S - 1) * nodes * N * cs);
    a->off_v = align256(a->off_a + S * nodes * N * cs);
    a->off_g = align256(a->off_v + S * nodes * N * cs);
    a->off_gx = align256(a->off_g + nodes * N * cs);
    a->off_gs = align256(a->off_gx + N * sizeof(double2));
    a->off_p0 = align256(a->off_gs + N * sizeof(double2));
    a->off_part = align256(a->off_p0 + N * cs);
    a->off_acc = align256(a->off_part + (size_t)a->tiles * sizeof(double));
    a->off_adjc = align256(a->off_acc + (size_t)a->n_int * a->acc_stride * sizeof(double));
    a->need = align256(a->off_adjc + (size_t)p->n_types * nodes * sizeof(AdjC));
    return MPA_OK;
}

// Physical segment (p n_seg + s) holding z from the left (sgn < 0) or the
// right (sgn > 0), the same side convention as HostMap::side; -1 outside.
int seg_index(const HostMap& m, double z, int sgn) {
    const double zz = z + (sgn > 0 ? 1e-9 : -1e-9) * m.period;
    const long per = (long)std::floor(zz / m.period);
    const double u = zz - (double)per * m.period;
    double a = 0.0;
    int s = (int)m.seg.size() - 1;
    for (size_t i = 0; i < m.seg.size(); ++i) {
        a += m.seg[i].length_km;
        if (u < a) {
            s = (int)i;
            break;
        }
    }
    if (per < 0 || per >= n_periods_of(m)) return -1;
    return (int)per * (int)m.seg.size() + s;
}

// g[P] += w |[za, zb] n segment P| over the physical segments.
void add_overlaps(const HostMap& m, double za, double zb, double w, double* g) {
    if (!(zb > za) || w == 0.0 || !g) return;
    const int np = n_periods_of(m);
    const long p0 = std::max(0L, (long)std::floor(za / m.period) - 1);
    const long p1 = std::min((long)np - 1, (long)std::floor(zb / m.period) + 1);
    for (long per = p0; per <= p1; ++per) {
        double a = (double)per * m.period;
        for (size_t i = 0; i < m.seg.size(); ++i) {
            const double b = a + m.seg[i].length_km;
            const double lo = a > za ? a : za, hi = b < zb ? b : zb;
            if (hi > lo) g[per * (long)m.seg.size() + (long)i] += w * (hi - lo);
            a = b;
        }
    }
}

// Per-node constants of the reverse pass for every interval type: the same
// dz, loss factor and sigma(z_j) as the plan's node table.
std::vector<AdjC> adj_table(const mpa_plan* p) {
    const int M = p->M;
    const double dz = p->L / M;
    std::vector<AdjC> v((size_t)p->n_types * (M + 1));
    for (int t = 0; t < p->n_types; ++t) {
        const double u0 = p->L * t;
        for (int j = 0; j <= M; ++j) {
            const double zr = (j == M) ? p->L : dz * j;
            double sig;
            if (j == 0) sig = p->map.side(u0, 3, +1);
            else if (j == M) sig = p->map.side(u0 + zr, 3, -1);
            else sig = 0.5 * (p->map.side(u0 + zr, 3, -1) + p->map.side(u0 + zr, 3, +1));
            AdjC& c = v[(size_t)t * (M + 1) + j];
            c.dzp = dz / std::exp(p->map.G(u0, u0 + zr));
            c.sig = sig;
        }
    }
    return v;
}

// A_hat(z_from) = F[field] into the plan's state, then the intervals, storing
// the state before each interval and the final one (n_int + 1 checkpoints);
// if out is non-null it receives A(z_to).
template <typename T>
int forward_ckpt(mpa_plan* p, const void* field, const AdjLayout& a, double2* ck, void* out, cudaStream_t st) {
    const Split& s = p->sp;
    const size_t N = (size_t)s.N;
    cx<T>* psi = reinterpret_cast<cx<T>*>(p->ws + p->off_psi);
    double2* state = reinterpret_cast<double2*>(p->ws + p->off_state);
    cx<T>* psi0c = reinterpret_cast<cx<T>*>(p->ws + p->off_psi0c);
    int rc = fft_forward<T>(s, reinterpret_cast<const cx<T>*>(field), psi, st);
    if (rc) return rc;
    MPA_TRY(to_state_launch<T>(psi, state, sizeof(T) == 4 ? psi0c : nullptr, s.N, st));
    for (long q = 0; q < a.n_int; ++q) {
        MPA_TRY(cudaMemcpyAsync(ck + (size_t)q * N, state, N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        rc = run_interval<T>(p, a.types[(size_t)q], a.amps[(size_t)q], 1, nullptr, st);
        if (rc) return rc;
    }
    MPA_TRY(cudaMemcpyAsync(ck + (size_t)a.n_int * N, state, N * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    if (out) {
        MPA_TRY(from_state_launch<T>(state, psi, s.N, st));
        return fft_inverse<T>(s, psi, reinterpret_cast<cx<T>*>(out), st);
    }
    return MPA_OK;
}

template <typename T>
int adjoint_t(mpa_plan* p, const void* field_in, const void* grad_out, void* grad_in, const AdjLayout& a,
              unsigned char* ws, double* grad_sigma, double* grad_beta2, cudaStream_t st) {
    typedef cx<T> C;
    const Split& s = p->sp;
    const long long N = s.N;
    const int M = p->M, S = p->n_iter, nodes = M + 1;
    const size_t NM = (size_t)nodes * (size_t)N;
    double2* ck = reinterpret_cast<double2*>(ws + a.off_ck);
    C* psi_lv = reinterpret_cast<C*>(ws + a.off_psi);  // psi^{(n)}, n = 1..S-1
    C* a_lv = reinterpret_cast<C*>(ws + a.off_a);      // A^{(n)}(t), n = 0..S-1 (row pass layout)
    C* v_lv = reinterpret_cast<C*>(ws + a.off_v);      // V^{(n)}, n = 0..S-1
    C* G = reinterpret_cast<C*>(ws + a.off_g);
    double2* gx = reinterpret_cast<double2*>(ws + a.off_gx);
    double2* gs = reinterpret_cast<double2*>(ws + a.off_gs);
    C* p0 = reinterpret_cast<C*>(ws + a.off_p0);
    double* part = reinterpret_cast<double*>(ws + a.off_part);
    double* acc = reinterpret_cast<double*>(ws + a.off_acc);
    AdjC* adjc = reinterpret_cast<AdjC*>(ws + a.off_adjc);
    C* W = reinterpret_cast<C*>(p->ws + p->off_psi);
    const NodeC* nodes_d = reinterpret_cast<const NodeC*>(p->ws + p->off_nodes);
    const int* toff = reinterpret_cast<const int*>(p->ws + p->off_toff);
    auto psi_slot = [&](int n) { return psi_lv + (size_t)(n - 1) * NM; };
    const double wscale = 0.5 * (2.0 * kPi / p->T) * (2.0 * kPi / p->T);
    const int gc = kca_tile_cols<T>(s.logN2), gr = kra_tile_rows<T>(s.logN1);
    const int kc_per = (int)(s.N1 / gc), kr_per = (int)(s.N2 / gr);

    if (field_in) {
        int rc = forward_ckpt<T>(p, field_in, a, ck, nullptr, st);
        if (rc) return rc;
    }
    const std::vector<AdjC> tab = adj_table(p);
    MPA_TRY(cudaMemcpyAsync(adjc, tab.data(), tab.size() * sizeof(AdjC), cudaMemcpyHostToDevice, st));
    MPA_TRY(cudaMemsetAsync(acc, 0, (size_t)a.n_int * a.acc_stride * sizeof(double), st));
    // A_out = F^-1[A_hat]  =>  g_{A_hat} = F[g_out] / N
    int rc = fft_forward<T>(s, reinterpret_cast<const C*>(grad_out), G, st);
    if (rc) return rc;
    MPA_TRY(scale_to_state_launch<T>(G, gx, 1.0 / (double)N, N, st));

    auto kc_pre = [&](int n, int t) {
        KCParams<T> c{};
        c.src = n == 0 ? p0 : psi_slot(n);
        c.src_stride = n == 0 ? 0 : N;
        c.dst = W;
        c.dst_stride = N;
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.ncols = (long long)nodes * s.N1;
        c.npl = nodes;
        c.nodes = nodes_d;
        c.loff = toff + t;
        return kc_launch<T>(KC_MPA_PRE, s.logN2, c, st);
    };
    auto kca = [&](int mode, int n, int t, double* accq) {
        KCAParams<T> c{};
        c.g = G;
        if (mode == KCA_G) {
            c.aux = v_lv + (size_t)n * NM;
            c.aux_stride = N;
        } else {
            c.aux = n == 0 ? p0 : psi_slot(n);
            c.aux_stride = n == 0 ? 0 : N;
        }
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.ncols = (long long)nodes * s.N1;
        c.nodes = nodes_d + (size_t)t * nodes;
        c.adj = adjc + (size_t)t * nodes;
        c.wscale = wscale;
        c.part = part;
        cudaError_t e = kca_launch<T>(mode, s.logN2, c, st);
        if (e == cudaSuccess) e = reduce_parts_launch(part, kc_per, nodes, accq, st);
        return e;
    };

    for (long q = a.n_int - 1; q >= 0; --q) {
        const int t = a.types[(size_t)q];
        double* accq = acc + (size_t)q * a.acc_stride;
        MPA_TRY(from_state_launch<T>(ck + (size_t)q * N, p0, N, st));
        // recompute the levels of this interval, every one kept
        for (int n = 0; n < S; ++n) {
            MPA_TRY(kc_pre(n, t));
            KRParams<T> r{W, (long long)nodes * s.N2, N, s.logN, (int)s.N2, (T)(1.0 / (double)N), T(0)};
            r.keep = a_lv + (size_t)n * NM;
            MPA_TRY(kr_keep_launch<T>(s.logN1, r, st));
            KCParams<T> c{};
            c.src = W;
            c.src_stride = N;
            c.dst = v_lv + (size_t)n * NM;
            c.dst_stride = N;
            c.N = N;
            c.logN = s.logN;
            c.N1 = (int)s.N1;
            c.logN1 = s.logN1;
            c.ncols = (long long)nodes * s.N1;
            c.npl = nodes;
            c.nodes = nodes_d;
            c.loff = toff + t;
            MPA_TRY(kc_launch<T>(KC_MPA_POST, s.logN2, c, st));
            if (n + 1 < S) MPA_TRY(scan_store_launch<T>(v_lv + (size_t)n * NM, psi_slot(n + 1), p0, N, M, st));
        }
        // step 7 and the last level's step 5, reversed
        MPA_TRY(cudaMemsetAsync(gs, 0, (size_t)N * sizeof(double2), st));
        RScanParams<T> rs{};
        rs.g = G;
        rs.gs0 = gs;
        rs.N = N;
        rs.M = M;
        rs.mode = RSCAN_TOP;
        rs.gX = gx;
        rs.X = ck + (size_t)(q + 1) * N;
        rs.nodeM = p->nodes[(size_t)t * nodes + M];
        rs.scaleM = rs.nodeM.pre * std::exp((double)a.amps[(size_t)q] * p->map.z_a * p->map.gamma);
        rs.wscale = wscale;
        rs.part = part;
        MPA_TRY(rscan_launch<T>(rs, st));
        MPA_TRY(reduce_parts_launch(part, (int)((N + 255) / 256), 1, accq + 2 * nodes, st));
        for (int n = S - 1; n >= 0; --n) {
            if (n + 1 < S) {
                rs.mode = RSCAN_LEVEL;
                MPA_TRY(rscan_launch<T>(rs, st));
            }
            MPA_TRY(kca(KCA_G, n, t, accq));
            KRAParams<T> r{};
            r.a = a_lv + (size_t)n * NM;
            r.g = G;
            r.nrows = (long long)nodes * s.N2;
            r.N = N;
            r.logN = s.logN;
            r.N2 = (int)s.N2;
            r.adj = adjc + (size_t)t * nodes;
            r.part = part;
            MPA_TRY(kra_launch<T>(s.logN1, r, st));
            MPA_TRY(reduce_parts_launch(part, kr_per, nodes, accq + nodes, st));
            MPA_TRY(kca(KCA_P, n, t, accq));
        }
        // psi^{(0)}_j = psi_0 at every node
        rs.mode = RSCAN_SUM;
        MPA_TRY(rscan_launch<T>(rs, st));
        std::swap(gx, gs);
    }
    // A_hat(z_from) = F[A_in]  =>  g_{A_in} = N F^-1[g_{A_hat}] (the unscaled inverse)
    MPA_TRY(from_state_launch<T>(gx, G, N, st));
    {
        KCParams<T> c{};
        c.src = G;
        c.dst = G;
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.ncols = s.N1;
        MPA_TRY(kc_launch<T>(KC_INV, s.logN2, c, st));
        KRParams<T> r{G, s.N2, N, s.logN, (int)s.N2, T(1), T(0)};
        MPA_TRY(kr_launch<T>(KR_INV, s.logN1, r, st));
        MPA_TRY(transpose_launch<T>(G, reinterpret_cast<C*>(grad_in), s.N2, s.N1, st));
    }
    if (!grad_sigma && !grad_beta2) return MPA_OK;
    std::vector<double> h((size_t)a.n_int * a.acc_stride);
    MPA_TRY(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MPA_TRY(cudaStreamSynchronize(st));
    const HostMap& m = p->map;
    const int n_phys = n_periods_of(m) * (int)m.seg.size();
    std::vector<double> gsig((size_t)n_phys, 0.0), gb2((size_t)n_phys, 0.0);
    const double dz = p->L / M;
    for (long q = 0; q < a.n_int; ++q) {
        const double z0 = a.z_from + p->L * (double)q;
        const double* b = h.data() + (size_t)q * a.acc_stride;
        for (int j = 0; j <= M; ++j) {
            const double zj = (j == M) ? z0 + p->L : z0 + dz * j;
            add_overlaps(m, z0, zj, b[j], gb2.data());
            const double hs = b[nodes + j];
            const int sl = seg_index(m, zj, -1), sr = seg_index(m, zj, +1);
            if (j == 0) {
                if (sr >= 0) gsig[(size_t)sr] += hs;
            } else if (j == M) {
                if (sl >= 0) gsig[(size_t)sl] += hs;
            } else {
                if (sl >= 0) gsig[(size_t)sl] += 0.5 * hs;
                if (sr >= 0) gsig[(size_t)sr] += 0.5 * hs;
            }
        }
        add_overlaps(m, z0, z0 + p->L, b[2 * nodes], gb2.data());
    }
    if (grad_sigma) std::copy(gsig.begin(), gsig.end(), grad_sigma);
    if (grad_beta2) std::copy(gb2.begin(), gb2.end(), grad_beta2);
    return MPA_OK;
}

int check_ws(const AdjLayout& a, void* ws, size_t bytes) {
    if (!ws || bytes < a.need || ((uintptr_t)ws & 255u) != 0) return MPA_ERR_WORKSPACE;
    return MPA_OK;
}

}  // namespace

namespace mpa {

// acc[i] += sum_{t < per} part[i per + t], in order (deterministic).
__global__ void __launch_bounds__(128) reduce_parts_kernel(const double* __restrict__ part, int per, int n,
                                                           double* __restrict__ acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int t = 0; t < per; ++t) s += part[(long long)i * per + t];
    acc[i] += s;
}

cudaError_t reduce_parts_launch(const double* part, int per, int n, double* acc, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    reduce_parts_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(part, per, n, acc);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mpa

extern "C" {

int mpa_plan_n_segments(const mpa_plan* p, int32_t* n) {
    if (!p || !n) return MPA_ERR_INVALID_ARG;
    *n = (int32_t)(n_periods_of(p->map) * (int)p->map.seg.size());
    return MPA_OK;
}

int mpa_adjoint_workspace_size(const mpa_plan* p, double z_from_km, double z_to_km, size_t* bytes) {
    return abi_call([&]() -> int {
        if (!p || !bytes) return MPA_ERR_INVALID_ARG;
        AdjLayout a;
        const int rc = adj_layout(p, z_from_km, z_to_km, &a);
        if (rc) return rc;
        *bytes = a.need;
        return MPA_OK;
    });
}

int mpa_propagate_checkpointed(mpa_plan* p, void* field, double z_from_km, double z_to_km, void* adj_ws,
                               size_t adj_bytes, mpa_stream stream) {
    return abi_call([&]() -> int {
        mpa::host::EntryRange nv("mpa_propagate_checkpointed", stream);
        if (!p || !field) return MPA_ERR_INVALID_ARG;
        if (!p->ws) return MPA_ERR_WORKSPACE;
        AdjLayout a;
        int rc = adj_layout(p, z_from_km, z_to_km, &a);
        if (rc) return rc;
        if ((rc = check_ws(a, adj_ws, adj_bytes))) return rc;
        double2* ck = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(adj_ws) + a.off_ck);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        return p->prec == MPA_FP32 ? forward_ckpt<float>(p, field, a, ck, field, st)
                                   : forward_ckpt<double>(p, field, a, ck, field, st);
    });
}

int mpa_adjoint(mpa_plan* p, const void* field_in, const void* grad_out, void* grad_in, double z_from_km,
                double z_to_km, void* adj_ws, size_t adj_bytes, double* grad_sigma, double* grad_beta2,
                mpa_stream stream) {
    return abi_call([&]() -> int {
        mpa::host::EntryRange nv("mpa_adjoint", stream);
        if (!p || !grad_out || !grad_in) return MPA_ERR_INVALID_ARG;
        if (!p->ws) return MPA_ERR_WORKSPACE;
        AdjLayout a;
        int rc = adj_layout(p, z_from_km, z_to_km, &a);
        if (rc) return rc;
        if ((rc = check_ws(a, adj_ws, adj_bytes))) return rc;
        unsigned char* ws = reinterpret_cast<unsigned char*>(adj_ws);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        if (p->prec == MPA_FP32) return adjoint_t<float>(p, field_in, grad_out, grad_in, a, ws, grad_sigma, grad_beta2, st);
        return adjoint_t<double>(p, field_in, grad_out, grad_in, a, ws, grad_sigma, grad_beta2, st);
    });
}

}  // extern "C"
