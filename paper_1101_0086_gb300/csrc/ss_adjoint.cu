// Reverse mode of ss_propagate (the split-step of Eq. (4)): gradients of a
// real loss with respect to the input field and to sigma and beta2 of every
// physical segment.
//
// Schedule: a forward pass keeps the working buffer every Kc steps
// (checkpoints, working precision, the permuted four-step layout the
// split-step kernels pass between them).  The segments of Kc steps are then
// walked backwards: each is recomputed from its checkpoint with the
// time-domain field before every nonlinear step and the spectrum after every
// linear step kept (adjoint.cuh, SSR/SSC STORE), then reversed step by step
// (SSC/SSR REV).  The parameter sums of every step go to a device table that
// the host folds into the segments.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "adj_launch.h"
#include "host.h"

using namespace mpa;
using namespace mpa::host;

namespace {

struct SSAdj {
    long K = 0;        // steps
    long Kc = 0;       // steps per checkpoint segment
    long n_ck = 0;     // checkpoints
    long long tiles_c = 0, tiles_r = 0;
    size_t off_ck = 0, off_t = 0, off_x = 0, off_w = 0, off_g = 0, off_pb = 0, off_ps = 0, off_acc = 0, need = 0;
};

int ss_layout(const HostMap& m, const Split& s, int prec, double dz, double z_from, double z_to, int ckpt_steps,
              SSAdj* a) {
    double kk;
    if (!(z_from >= -1e-12) || !(z_to > z_from) || z_to > m.length * (1 + 1e-12) + 1e-9) return MPA_ERR_GRID;
    if (!whole((z_to - z_from) / dz, &kk) || kk < 1 || kk > kMaxIntervals) return MPA_ERR_GRID;
    if (s.logN < 13) return MPA_ERR_UNSUPPORTED_N;
    a->K = (long)kk;
    a->Kc = ckpt_steps > 0 ? ckpt_steps : (long)std::ceil(std::sqrt((double)a->K));
    if (a->Kc > a->K) a->Kc = a->K;
    a->n_ck = (a->K + a->Kc - 1) / a->Kc;
    const bool f32 = prec == MPA_FP32;
    const int gc = f32 ? kca_tile_cols<float>(s.logN2) : kca_tile_cols<double>(s.logN2);
    const int gr = f32 ? kra_tile_rows<float>(s.logN1) : kra_tile_rows<double>(s.logN1);
    if (gc <= 0 || gr <= 0 || gc > s.N1 || gr > s.N2) return MPA_ERR_UNSUPPORTED_N;
    a->tiles_c = s.N1 / gc;
    a->tiles_r = s.N2 / gr;
    const size_t N = (size_t)s.N, cs = f32 ? sizeof(float2) : sizeof(double2);
    a->off_ck = 0;
    a->off_t = align256(a->off_ck + (size_t)a->n_ck * N * cs);
    a->off_x = align256(a->off_t + (size_t)a->Kc * N * cs);
    a->off_w = align256(a->off_x + (size_t)(a->Kc + 1) * N * cs);
    a->off_g = align256(a->off_w + N * cs);
    a->off_pb = align256(a->off_g + N * cs);
    a->off_ps = align256(a->off_pb + (size_t)(a->Kc + 1) * a->tiles_c * sizeof(double));
    a->off_acc = align256(a->off_ps + (size_t)a->Kc * a->tiles_r * sizeof(double));
    a->need = align256(a->off_acc + (size_t)(2 * a->K + 1) * sizeof(double));
    return MPA_OK;
}

int n_periods_of(const HostMap& m) { return (int)std::lround(m.length / m.period); }

void add_overlaps(const HostMap& m, double za, double zb, double w, double* g) {
    if (!(zb > za) || w == 0.0) return;
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

template <typename T>
int ss_adjoint_t(const HostMap& m, const Split& s, double T_ps, double dz, const void* field_in, const void* grad_out,
                 void* grad_in, double z_from, double z_to, const SSAdj& a, unsigned char* ws, double* grad_sigma,
                 double* grad_beta2, cudaStream_t st) {
    typedef cx<T> C;
    const long long N = s.N;
    const long K = a.K, Kc = a.Kc;
    C* ck = reinterpret_cast<C*>(ws + a.off_ck);
    C* tr = reinterpret_cast<C*>(ws + a.off_t);
    C* xs = reinterpret_cast<C*>(ws + a.off_x);
    C* w = reinterpret_cast<C*>(ws + a.off_w);
    C* g = reinterpret_cast<C*>(ws + a.off_g);
    double* pb = reinterpret_cast<double*>(ws + a.off_pb);
    double* ps = reinterpret_cast<double*>(ws + a.off_ps);
    double* acc = reinterpret_cast<double*>(ws + a.off_acc);  // K+1 linear steps, then K nonlinear steps
    const double wscale = 0.5 * (2.0 * kPi / T_ps) * (2.0 * kPi / T_ps);
    // the steps of Eq. (4) exactly as ss_propagate takes them
    auto lin = [&](long k, double* za, double* zb) {
        if (k == 0) {
            *za = z_from;
            *zb = z_from + 0.5 * dz;
        } else {
            *za = z_from + dz * (double)(k - 1) + 0.5 * dz;
            *zb = (k == K) ? z_to : *za + dz;
        }
    };
    auto flow = [&](long k, bool conj) {
        double za, zb;
        lin(k, &za, &zb);
        NodeC c{};
        const double I2 = m.integ(za, zb, 1), I3 = m.integ(za, zb, 2);
        phase_consts(conj ? -I2 : I2, conj ? -I3 : I3, T_ps, &c);
        c.pre = std::exp(m.G(za, zb) + (double)m.amps(za, zb) * m.z_a * m.gamma);
        c.post = 1.0;
        return c;
    };
    auto rot = [&](long k) {
        const double zk = z_from + dz * (double)k;
        return m.integ(zk, zk + dz, 3);
    };
    auto col = [&](int mode, C* data, long k, C* x, double* part, double scale) {
        SSCParams<T> c{};
        c.data = data;
        c.xs = x;
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.flow = flow(k, mode == SS_REV);
        c.pre = c.flow.pre * scale;
        c.wscale = wscale * scale;  // the beta2 sum uses the incoming gradient times scale
        c.part = part;
        return ssc_launch<T>(mode, s.logN2, c, st);
    };
    auto row = [&](int mode, C* data, long k, C* t, double* part) {
        SSRParams<T> r{};
        r.data = data;
        r.ts = t;
        r.nrows = s.N2;
        r.N = N;
        r.logN = s.logN;
        r.N2 = (int)s.N2;
        r.inv_n = (T)(1.0 / (double)N);
        r.rot = (T)rot(k);
        r.scale = (double)N;
        r.part = part;
        return ssr_launch<T>(mode, s.logN1, r, st);
    };
    auto entry = [&](const void* f, C* dst) -> int {
        MPA_TRY(transpose_launch<T>(reinterpret_cast<const C*>(f), dst, s.N1, s.N2, st));
        KRParams<T> r{dst, s.N2, N, s.logN, (int)s.N2, (T)(1.0 / (double)N), T(0)};
        MPA_TRY(kr_launch<T>(KR_FWD, s.logN1, r, st));
        return MPA_OK;
    };

    // forward with a checkpoint before steps 0, Kc, 2 Kc, ...
    int rc = entry(field_in, w);
    if (rc) return rc;
    {
        KCParams<T> c{};
        c.src = w;
        c.dst = w;
        c.N = N;
        c.logN = s.logN;
        c.N1 = (int)s.N1;
        c.logN1 = s.logN1;
        c.ncols = s.N1;
        c.flow = flow(0, false);
        MPA_TRY(kc_launch<T>(KC_SS_STEP, s.logN2, c, st));
        for (long k = 0; k < K; ++k) {
            if (k % Kc == 0)
                MPA_TRY(cudaMemcpyAsync(ck + (size_t)(k / Kc) * N, w, (size_t)N * sizeof(C), cudaMemcpyDeviceToDevice,
                                        st));
            KRParams<T> r{w, s.N2, N, s.logN, (int)s.N2, (T)(1.0 / (double)N), (T)rot(k)};
            MPA_TRY(kr_launch<T>(KR_SS, s.logN1, r, st));
            c.flow = flow(k + 1, false);
            MPA_TRY(kc_launch<T>(KC_SS_STEP, s.logN2, c, st));
        }
    }
    MPA_TRY(cudaMemsetAsync(acc, 0, (size_t)(2 * K + 1) * sizeof(double), st));
    // A_out = F^-1[X_K]: the reverse starts from F[g_out] / N (the 1/N is
    // applied with the last linear step)
    rc = entry(grad_out, g);
    if (rc) return rc;
    for (long seg = a.n_ck - 1; seg >= 0; --seg) {
        const long k0 = seg * Kc, k1 = std::min(K, k0 + Kc);
        // recompute: t_k before nonlinear step k at tr[k - k0], X' after linear step k at xs[k - k0]
        if (seg == 0) {
            rc = entry(field_in, w);
            if (rc) return rc;
            MPA_TRY(col(SS_STORE, w, 0, xs, nullptr, 1.0));
        } else {
            MPA_TRY(cudaMemcpyAsync(w, ck + (size_t)seg * N, (size_t)N * sizeof(C), cudaMemcpyDeviceToDevice, st));
        }
        for (long k = k0; k < k1; ++k) {
            MPA_TRY(row(SS_STORE, w, k, tr + (size_t)(k - k0) * N, nullptr));
            MPA_TRY(col(SS_STORE, w, k + 1, xs + (size_t)(k - k0 + 1) * N, nullptr, 1.0));
        }
        // reverse
        for (long k = k1 - 1; k >= k0; --k) {
            MPA_TRY(col(SS_REV, g, k + 1, xs + (size_t)(k - k0 + 1) * N, pb + (k - k0 + 1) * a.tiles_c,
                        k + 1 == K ? 1.0 / (double)N : 1.0));
            MPA_TRY(row(SS_REV, g, k, tr + (size_t)(k - k0) * N, ps + (k - k0) * a.tiles_r));
        }
        if (seg == 0) {
            MPA_TRY(col(SS_REV, g, 0, xs, pb, 1.0));
            MPA_TRY(reduce_parts_launch(pb, (int)a.tiles_c, 1, acc, st));
        }
        MPA_TRY(reduce_parts_launch(pb + a.tiles_c, (int)a.tiles_c, (int)(k1 - k0), acc + k0 + 1, st));
        MPA_TRY(reduce_parts_launch(ps, (int)a.tiles_r, (int)(k1 - k0), acc + (K + 1) + k0, st));
    }
    // X_0 = F[A_in]: g_A = N F^-1[g_X0] (unscaled inverse); the inverse
    // column pass ran inside the last reverse column pass
    KRParams<T> ri{g, s.N2, N, s.logN, (int)s.N2, T(1), T(0)};
    MPA_TRY(kr_launch<T>(KR_INV, s.logN1, ri, st));
    MPA_TRY(transpose_launch<T>(g, reinterpret_cast<C*>(grad_in), s.N2, s.N1, st));
    if (!grad_sigma && !grad_beta2) return MPA_OK;
    std::vector<double> h((size_t)(2 * K + 1));
    MPA_TRY(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MPA_TRY(cudaStreamSynchronize(st));
    const int n_phys = n_periods_of(m) * (int)m.seg.size();
    std::vector<double> gs((size_t)n_phys, 0.0), gb((size_t)n_phys, 0.0);
    for (long k = 0; k <= K; ++k) {
        double za, zb;
        lin(k, &za, &zb);
        add_overlaps(m, za, zb, h[(size_t)k], gb.data());
    }
    for (long k = 0; k < K; ++k) {
        const double zk = z_from + dz * (double)k;
        add_overlaps(m, zk, zk + dz, h[(size_t)(K + 1 + k)], gs.data());
    }
    if (grad_sigma) std::copy(gs.begin(), gs.end(), grad_sigma);
    if (grad_beta2) std::copy(gb.begin(), gb.end(), grad_beta2);
    return MPA_OK;
}

}  // namespace

extern "C" {

int ss_adjoint_workspace_size(const mpa_fiber_map* map, int64_t N, int32_t precision, double dz_km, double z_from_km,
                              double z_to_km, int32_t ckpt_steps, size_t* bytes) {
    return abi_call([&]() -> int {
        if (!map || !bytes || !(dz_km > 0.0)) return MPA_ERR_INVALID_ARG;
        if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
        HostMap m;
        int rc = m.init(map);
        if (rc) return rc;
        Split s;
        if ((rc = split_n(N, precision, &s))) return rc;
        SSAdj a;
        if ((rc = ss_layout(m, s, precision, dz_km, z_from_km, z_to_km, ckpt_steps, &a))) return rc;
        *bytes = a.need;
        return MPA_OK;
    });
}

int ss_adjoint(const mpa_fiber_map* map, int64_t N, double T_ps, double dz_km, int32_t precision, const void* field_in,
               const void* grad_out, void* grad_in, double z_from_km, double z_to_km, int32_t ckpt_steps,
               void* workspace, size_t ws_bytes, double* grad_sigma, double* grad_beta2, mpa_stream stream) {
    return abi_call([&]() -> int {
        mpa::host::EntryRange nv("ss_adjoint", stream);
        if (!map || !field_in || !grad_out || !grad_in || !(T_ps > 0.0) || !(dz_km > 0.0)) return MPA_ERR_INVALID_ARG;
        if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
        HostMap m;
        int rc = m.init(map);
        if (rc) return rc;
        Split s;
        if ((rc = split_n(N, precision, &s))) return rc;
        SSAdj a;
        if ((rc = ss_layout(m, s, precision, dz_km, z_from_km, z_to_km, ckpt_steps, &a))) return rc;
        if (!workspace || ws_bytes < a.need || ((uintptr_t)workspace & 255u) != 0) return MPA_ERR_WORKSPACE;
        unsigned char* ws = reinterpret_cast<unsigned char*>(workspace);
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        return precision == MPA_FP32
                   ? ss_adjoint_t<float>(m, s, T_ps, dz_km, field_in, grad_out, grad_in, z_from_km, z_to_km, a, ws,
                                         grad_sigma, grad_beta2, st)
                   : ss_adjoint_t<double>(m, s, T_ps, dz_km, field_in, grad_out, grad_in, z_from_km, z_to_km, a, ws,
                                          grad_sigma, grad_beta2, st);
    });
}

}  // extern "C"
