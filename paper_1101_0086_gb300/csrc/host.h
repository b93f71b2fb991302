// Host-side helpers shared by the single-link plan (plan.cu) and the
// batched links (batch.cu): fiber-map integration, the fixed-point phase
// constants, the four-step split of N, and the natural-order transforms.
#pragma once

#include <cmath>
#include <cstdlib>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "launch.h"
#include "mpa.h"

namespace mpa {
namespace host {

// NVTX range around an entry point or an interval (header-only NVTX3: a few
// nanoseconds when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// An entry point: its NVTX range and, while profiling is on, its per-call
// CUDA-event timer.
struct EntryRange {
    EntryRange(const char* name, mpa_stream stream) : nv(name), timer(name, reinterpret_cast<cudaStream_t>(stream)) {}
    NvtxRange nv;
    CallTimer timer;
};

// Records the CUDA error string for mpa_last_cuda_error.
int cuda_fail(cudaError_t e);

#define MPA_TRY(expr)                                            \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return ::mpa::host::cuda_fail(_e); \
    } while (0)

// Body of a C entry point: no C++ exception may cross the C ABI, so a host
// allocation that fails (or a container size beyond what the host can hold)
// becomes MPA_ERR_HOST_MEMORY and any other exception MPA_ERR_INVALID_ARG.
// Objects the body owns must be held by RAII (std::unique_ptr, containers)
// so that nothing leaks on that path.
template <class F> int abi_call(F&& body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc&) {
        return MPA_ERR_HOST_MEMORY;
    } catch (const std::length_error&) {
        return MPA_ERR_HOST_MEMORY;
    } catch (...) {
        return MPA_ERR_INVALID_ARG;
    }
}

inline constexpr double kPi = 3.14159265358979323846264338327950288;
// largest node count parameter M of a plan or batch (every size computed
// from M + 1 stays far inside 64 bits and M + 1 inside 32)
inline constexpr int kMaxNodes = 1 << 24;
// most distinct interval starts within one period (period / L), and most
// intervals of one link; larger counts are reported as MPA_ERR_GRID
inline constexpr double kMaxIntervalTypes = (double)(1 << 20);
inline constexpr double kMaxIntervals = 2147483647.0;
// default polls of each bounded wait of a persistent kernel (a few seconds
// at most; a wait normally ends within microseconds)
inline constexpr long long kSpinLimit = 1ll << 22;
// amplifiers that may end one interval (a longer interval than the
// amplifier spacing would cross one inside it, which is rejected)
inline constexpr int kMaxAmpsPerInterval = 4;

// ----------------------------------------------------------- fiber map
struct HostMap {
    std::vector<mpa_segment> seg;
    double gamma = 0, z_a = 0, period = 0, length = 0;

    int init(const mpa_fiber_map* m) {
        if (!m || !m->segments || m->n_segments < 1 || m->n_periods < 1) return MPA_ERR_INVALID_ARG;
        if (!(m->gamma_per_km >= 0.0) || !std::isfinite(m->gamma_per_km) || !std::isfinite(m->z_a_km))
            return MPA_ERR_INVALID_ARG;
        seg.assign(m->segments, m->segments + m->n_segments);
        for (const auto& s : seg) {
            if (!(s.length_km > 0.0) || !std::isfinite(s.beta2_ps2_per_km) || !std::isfinite(s.beta3_ps3_per_km) ||
                !std::isfinite(s.sigma_per_W_km) || !std::isfinite(s.gain_per_km))
                return MPA_ERR_INVALID_ARG;
            period += s.length_km;
        }
        gamma = m->gamma_per_km;
        z_a = m->z_a_km;
        length = period * m->n_periods;
        return MPA_OK;
    }
    // col 1: beta2, 2: beta3, 3: sigma, 4: distributed gain
    static double coef(const mpa_segment& s, int col) {
        return col == 1 ? s.beta2_ps2_per_km : col == 2 ? s.beta3_ps3_per_km : col == 3 ? s.sigma_per_W_km
                                                                                       : s.gain_per_km;
    }
    // int_za^zb of a coefficient: shift za into the first period, then sum
    // coefficient x overlap over the segment copies that [za, zb] covers.
    double integ(double za, double zb, int col) const {
        if (!(zb > za)) return 0.0;
        const double shift = std::floor(za / period) * period;
        const double u = za - shift, v = zb - shift;
        double acc = 0.0;
        for (long p = 0; (double)p * period < v; ++p) {
            double a = (double)p * period;
            for (const auto& s : seg) {
                const double b = a + s.length_km;
                const double lo = a > u ? a : u, hi = b < v ? b : v;
                if (hi > lo) acc += coef(s, col) * (hi - lo);
                a = b;
            }
        }
        return acc;
    }
    // coefficient just left (side < 0) or right (side > 0) of z
    double side(double z, int col, int sgn) const {
        const double zz = z + (sgn > 0 ? 1e-9 : -1e-9) * period;
        double u = zz - std::floor(zz / period) * period;
        double a = 0.0;
        for (size_t i = 0; i < seg.size(); ++i) {
            a += seg[i].length_km;
            if (u < a || i + 1 == seg.size()) return coef(seg[i], col);
        }
        return coef(seg.back(), col);
    }
    // int_za^zb G without the lumped amplifiers: the distributed gain minus gamma
    double G(double za, double zb) const { return integ(za, zb, 4) - gamma * (zb - za); }
    // amplifiers k z_a (k >= 1) in (za, zb]
    long amps(double za, double zb) const {
        if (!(z_a > 0.0)) return 0;
        const double tol = 1e-9 * z_a;
        long ka = (long)std::floor((za + tol) / z_a), kb = (long)std::floor((zb + tol) / z_a);
        if (ka < 0) ka = 0;
        return kb > ka ? kb - ka : 0;
    }
    // whether an amplifier z_k = k z_a (k >= 1) lies strictly inside
    // (za, zb), i.e. more than the tolerance of amps() away from both ends
    // (lumped gain is applied only at interval ends)
    bool amp_inside(double za, double zb) const {
        if (!(z_a > 0.0)) return false;
        const double tol = 1e-9 * z_a;
        long ka = (long)std::floor((za + tol) / z_a);        // k z_a > za + tol  <=>  k > ka
        const long kb = (long)std::ceil((zb - tol) / z_a) - 1;  // k z_a < zb - tol  <=>  k <= kb
        if (ka < 0) ka = 0;
        return kb > ka;
    }
};

// x mod 1 as a 128-bit binary fraction (exact whenever the FP64 value x has
// no bits below 2^-128).
inline void frac_q128(double x, unsigned long long* hi, unsigned long long* lo) {
    typedef unsigned __int128 u128;
    u128 q = 0;
    if (x != 0.0 && std::isfinite(x)) {
        const double ax = std::fabs(x);
        int e = 0;
        const double m = std::frexp(ax, &e);  // ax = m 2^e, m in [0.5, 1)
        const unsigned long long mant = (unsigned long long)std::ldexp(m, 53);
        const int sh = e - 53 + 128;  // ax 2^128 = mant 2^sh
        if (sh >= 128) q = 0;
        else if (sh >= 0) q = (u128)mant << sh;
        else if (sh > -64) q = (u128)(mant >> (-sh));
        if (x < 0) q = (u128)0 - q;
    }
    *hi = (unsigned long long)(q >> 64);
    *lo = (unsigned long long)q;
}

// Phase constants of beta(w, .) over an integral (I2, I3) for window T:
// theta = k'^2 pi I2/T^2 + k'^3 2 pi^2 I3/(3 T^3) turns.
inline void phase_consts(double I2, double I3, double T, NodeC* c) {
    frac_q128(kPi * I2 / (T * T), &c->a_hi, &c->a_lo);
    frac_q128(2.0 * kPi * kPi * I3 / (3.0 * T * T * T), &c->b_hi, &c->b_lo);
}

inline bool whole(double x, double* r) {
    const double n = std::nearbyint(x);
    *r = n;
    return std::fabs(x - n) <= 1e-9 * (std::fabs(x) > 1.0 ? std::fabs(x) : 1.0);
}

inline int ilog2(long long n) {
    int l = 0;
    while ((1ll << l) < n) ++l;
    return l;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

#ifndef MPA_LOGN2_SHIFT
#define MPA_LOGN2_SHIFT 0
#endif

struct Split {
    int logN, logN1, logN2;
    long long N, N1, N2;
    // node transforms of the MPA levels on chip (kn_kernel, one node per
    // tile row) instead of the column, row and column passes; N1 x N2 stays
    // the split of the entry/exit transforms and of the reverse mode
    bool onchip = false;
};

// Whether N fits the on-chip node transform in this precision.
inline bool onchip_ok(long long N, int prec) {
    const int l = ilog2(N);
    return (1ll << l) == N && l >= KN_LOG_MIN && l <= (prec == MPA_FP32 ? kn_log_max<float>() : kn_log_max<double>());
}

// The split with column length 2^logN2 (0 if the passes do not support it).
inline int split_with(long long N, int prec, int logN2, Split* s) {
    if (N < 256 || (N & (N - 1)) != 0) return MPA_ERR_UNSUPPORTED_N;
    s->logN = ilog2(N);
    s->logN2 = logN2;
    s->logN1 = s->logN - logN2;
    const int rmax = prec == MPA_FP32 ? kr_log_max<float>() : kr_log_max<double>();
    if (logN2 < KC_LOG_MIN || logN2 > KC_LOG_MAX || s->logN1 < KR_LOG_MIN || s->logN1 > rmax)
        return MPA_ERR_UNSUPPORTED_N;
    s->N = N;
    s->N1 = 1ll << s->logN1;
    s->N2 = 1ll << s->logN2;
    return MPA_OK;
}

inline int split_n(long long N, int prec, Split* s) {
    if (N < 256 || (N & (N - 1)) != 0) return MPA_ERR_UNSUPPORTED_N;
    s->logN = ilog2(N);
    if (s->logN > (prec == MPA_FP32 ? 25 : 24)) return MPA_ERR_UNSUPPORTED_N;
    // column length N2 = 2^logN2: about sqrt(N), shifted towards longer rows
    // by MPA_LOGN2_SHIFT (rows are contiguous, columns strided)
    int l2 = s->logN / 2 - MPA_LOGN2_SHIFT;
    if (l2 < KC_LOG_MIN) l2 = KC_LOG_MIN;
    if (l2 > KC_LOG_MAX) l2 = KC_LOG_MAX;
    s->logN2 = l2;
    s->logN1 = s->logN - s->logN2;
    const int rmax = prec == MPA_FP32 ? kr_log_max<float>() : kr_log_max<double>();
    if (s->logN2 < KC_LOG_MIN || s->logN1 > rmax) return MPA_ERR_UNSUPPORTED_N;
    s->N = N;
    s->N1 = 1ll << s->logN1;
    s->N2 = 1ll << s->logN2;
    return MPA_OK;
}

// ------------------------------------------------ natural-order transforms
// Forward: natural A(t) in `data` -> natural spectrum in `out` (may alias
// scratch); data viewed as N1 x N2 (rows n1), transposed into scratch.
template <typename T>
inline int fft_forward(const Split& s, const cx<T>* data, cx<T>* scratch, cudaStream_t st) {
    MPA_TRY(transpose_launch<T>(data, scratch, s.N1, s.N2, st));
    KRParams<T> r{scratch, s.N2, s.N, s.logN, (int)s.N2, (T)(1.0 / (double)s.N), T(0)};
    MPA_TRY(kr_launch<T>(KR_FWD, s.logN1, r, st));
    KCParams<T> c{};
    c.src = scratch;
    c.dst = scratch;
    c.N = s.N;
    c.logN = s.logN;
    c.N1 = (int)s.N1;
    c.logN1 = s.logN1;
    c.ncols = s.N1;
    MPA_TRY(kc_launch<T>(KC_FWD, s.logN2, c, st));
    return MPA_OK;
}

// Inverse: natural spectrum in `spec` (overwritten) -> natural A(t) in `out`.
template <typename T>
inline int fft_inverse(const Split& s, cx<T>* spec, cx<T>* out, cudaStream_t st) {
    KCParams<T> c{};
    c.src = spec;
    c.dst = spec;
    c.N = s.N;
    c.logN = s.logN;
    c.N1 = (int)s.N1;
    c.logN1 = s.logN1;
    c.ncols = s.N1;
    MPA_TRY(kc_launch<T>(KC_INV, s.logN2, c, st));
    KRParams<T> r{spec, s.N2, s.N, s.logN, (int)s.N2, (T)(1.0 / (double)s.N), T(0)};
    MPA_TRY(kr_launch<T>(KR_INV, s.logN1, r, st));
    MPA_TRY(transpose_launch<T>(spec, out, s.N2, s.N1, st));
    return MPA_OK;
}

// One level-synchronous interval (MPA steps 2-7) for nl links stored
// link-major; defined in plan.cu for float and double.  `work` (may be null)
// is a second set of node buffers of psi's size: with it, FP32 levels whose
// column passes run staged keep the node spectra in psi in the tile layout
// of the staged column pass and transform in `work` (a pass that changes
// the layout cannot work in place).
template <typename T>
int mpa_levels(const Split& s, int M, int n_iter, int nl, cx<T>* psi, cx<T>* work, cx<T>* psi0c, double2* state,
               const NodeC* nodes, const int* loff, const double* gain, const Monitor& mon, int scan_mode,
               double2* out, cudaStream_t st);
// Whether a plan or batch group of N modes in this precision gets the
// second set of node buffers (the staged column passes need N1 >= 32).
inline bool wants_work_buffers(long long N, int prec) { return prec == MPA_FP32 && N >= (1ll << 13); }

// Relative Picard increment below which a non-shrinking increment is
// rounding noise of the node-M sums rather than divergence.
inline constexpr double kDivergenceFloor = 1e-5;

}  // namespace host
}  // namespace mpa
