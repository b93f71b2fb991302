// Device building blocks of the MPA node transform and the split-step step:
// complex arithmetic, fixed-size DFTs in registers, the exact fixed-point
// dispersion phase, and a batched self-sorting (Stockham) FFT over shared
// memory.
//
// Fourier convention (text after Eq. (1)): forward F uses exp(+2 pi i kn/N)
// (sign S = +1), the inverse exp(-2 pi i kn/N) (S = -1, 1/N applied by the
// caller).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpa {

template <typename T> struct cx_of;
template <> struct cx_of<float> { typedef float2 type; };
template <> struct cx_of<double> { typedef double2 type; };
template <typename T> using cx = typename cx_of<T>::type;

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }

// FP32 complex add, subtract and real scaling as one packed f32x2
// instruction each (sm_100 and later): the same IEEE results as two scalar
// operations, half the issue slots.  MPA_F32X2=0 keeps the scalar forms.
#ifndef MPA_F32X2
#define MPA_F32X2 1
#endif
// packed real scalings (neutral in time, fewer instructions: on) and the
// cos/sin series of the phase in the two lanes of packed FMAs (slowed the
// forward column pass from 3.8 to 3.3-3.5 TB/s: off)
#ifndef MPA_F32X2_SCALE
#define MPA_F32X2_SCALE 1
#endif
#ifndef MPA_F32X2_POLY
#define MPA_F32X2_POLY 0
#endif
#if MPA_F32X2
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_from(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
// lane-wise a * b and a * b + c
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from(r);
}
#endif
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __device__ __forceinline__ C cconj(C a) { return mkc(a.x, -a.y); }
template <class C, class T> __device__ __forceinline__ C cscale(C a, T s) { return mkc(a.x * s, a.y * s); }
#if MPA_F32X2 && MPA_F32X2_SCALE
template <> __device__ __forceinline__ float2 cscale<float2, float>(float2 a, float s) { return mul2(a, make_float2(s, s)); }
#endif
// a * (S i)
template <int S, class C> __device__ __forceinline__ C mul_si(C a) {
    return S > 0 ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}
// a * exp(S i theta) given c = (cos, sin) of theta
template <int S, class C> __device__ __forceinline__ C mul_dir(C a, C w) {
    return S > 0 ? cmul(a, w) : cmul(a, cconj(w));
}

// ------------------------------------------------------------------ DFTs
// cos and sin of multiples of 2 pi/32 (closed forms: cos(pi/4) = sqrt(2)/2,
// cos(pi/8) = sqrt(2+sqrt(2))/2, sin(pi/8) = sqrt(2-sqrt(2))/2,
// cos(pi/16) = sqrt(2+sqrt(2+sqrt(2)))/2, sin(pi/16) = sqrt(2-sqrt(2+sqrt(2)))/2,
// cos(3pi/16) = sqrt(2+sqrt(2-sqrt(2)))/2, sin(3pi/16) = sqrt(2-sqrt(2-sqrt(2)))/2).
#define MPA_COS_PI_4 0.70710678118654752440
#define MPA_COS_PI_8 0.92387953251128675613
#define MPA_SIN_PI_8 0.38268343236508977173
#define MPA_COS_PI_16 0.98078528040323044913
#define MPA_SIN_PI_16 0.19509032201612826785
#define MPA_COS_3PI_16 0.83146961230254523708
#define MPA_SIN_3PI_16 0.55557023301960222474

// (cos, sin) of 2 pi m/32 for 0 < m < 16, m not a multiple of 4
template <int M32> struct Cs32 {
    static constexpr double c = (M32 == 1) ? MPA_COS_PI_16 : (M32 == 2) ? MPA_COS_PI_8 : (M32 == 3) ? MPA_COS_3PI_16
                              : (M32 == 5) ? MPA_SIN_3PI_16 : (M32 == 6) ? MPA_SIN_PI_8 : (M32 == 7) ? MPA_SIN_PI_16
                              : (M32 == 9) ? -MPA_SIN_PI_16 : (M32 == 10) ? -MPA_SIN_PI_8 : (M32 == 11) ? -MPA_SIN_3PI_16
                              : (M32 == 13) ? -MPA_COS_3PI_16 : (M32 == 14) ? -MPA_COS_PI_8 : -MPA_COS_PI_16;
    static constexpr double s = (M32 == 1) ? MPA_SIN_PI_16 : (M32 == 2) ? MPA_SIN_PI_8 : (M32 == 3) ? MPA_SIN_3PI_16
                              : (M32 == 5) ? MPA_COS_3PI_16 : (M32 == 6) ? MPA_COS_PI_8 : (M32 == 7) ? MPA_COS_PI_16
                              : (M32 == 9) ? MPA_COS_PI_16 : (M32 == 10) ? MPA_COS_PI_8 : (M32 == 11) ? MPA_COS_3PI_16
                              : (M32 == 13) ? MPA_SIN_3PI_16 : (M32 == 14) ? MPA_SIN_PI_8 : MPA_SIN_PI_16;
};

// v * exp(S 2 pi i K/R), R <= 32, 0 <= K < R/2 (compile-time special cases)
template <int R, int K, int S, class C> __device__ __forceinline__ C tw_const(C v) {
    typedef decltype(v.x) T;
    constexpr int M32 = K * (32 / R);
    if constexpr (M32 == 0) {
        return v;
    } else if constexpr (M32 == 8) {
        return mul_si<S>(v);
    } else if constexpr (M32 == 4 || M32 == 12) {
        const T c = (T)MPA_COS_PI_4;
        constexpr T re = (M32 == 4) ? T(1) : T(-1);
        // (re + S i) c
        return mkc(c * (re * v.x - T(S) * v.y), c * (re * v.y + T(S) * v.x));
    } else {
        const T cr = (T)Cs32<M32>::c, si = T(S) * (T)Cs32<M32>::s;
        return mkc(v.x * cr - v.y * si, v.x * si + v.y * cr);
    }
}

// FP32 butterflies with a non-trivial constant twiddle (K/R not a multiple
// of 1/4) as fused multiply-adds: x0 = e + w o with the twiddle's products
// folded into the additions, x1 = 2 e - x0 (= e - w o): six FP32 operations
// instead of eight (two products, two fused products and four additions).
// The difference from x1 = e - w o is one rounding of x0, of the size of the
// rounding of the product itself.  MPA_FMA_BFLY=0 keeps the plain form.
#ifndef MPA_FMA_BFLY
#define MPA_FMA_BFLY 1
#endif
template <int R, int K, int S> __device__ __forceinline__ void bfly_tw(float2& x0, float2& x1, float2 e, float2 o) {
    constexpr int M32 = K * (32 / R);
    float ax, ay;
    if constexpr (M32 == 4 || M32 == 12) {
        // w = c (re + S i), c = cos(pi/4): x0 = e + c (re o.x - S o.y, re o.y + S o.x)
        constexpr float re = (M32 == 4) ? 1.f : -1.f;
        const float c = (float)MPA_COS_PI_4;
        ax = fmaf(c, re * o.x - float(S) * o.y, e.x);
        ay = fmaf(c, re * o.y + float(S) * o.x, e.y);
    } else {
        const float cr = (float)Cs32<M32>::c, si = float(S) * (float)Cs32<M32>::s;
        ax = fmaf(o.x, cr, fmaf(-o.y, si, e.x));
        ay = fmaf(o.x, si, fmaf(o.y, cr, e.y));
    }
    x0 = make_float2(ax, ay);
    x1 = make_float2(fmaf(2.f, e.x, -ax), fmaf(2.f, e.y, -ay));
}

template <int R, int S, int K, class C> __device__ __forceinline__ void dft_combine(C* x, const C* e, const C* o) {
    if constexpr (K < R / 2) {
        constexpr int M32 = K * (32 / R);
        if constexpr (MPA_FMA_BFLY && sizeof(C) == 8 && M32 != 0 && M32 != 8) {
            bfly_tw<R, K, S>(x[K], x[K + R / 2], e[K], o[K]);
        } else {
            const C t = tw_const<R, K, S>(o[K]);
            x[K] = cadd(e[K], t);
            x[K + R / 2] = csub(e[K], t);
        }
        dft_combine<R, S, K + 1>(x, e, o);
    }
}

// In-register DFT of R points (power of two <= 32): X_k = sum_r x_r W^{rk},
// W = exp(S 2 pi i / R), by even/odd splitting.
template <int R, int S, class C> struct Dft {
    static __device__ __forceinline__ void run(C* x) {
        C e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = x[2 * i];
            o[i] = x[2 * i + 1];
        }
        Dft<R / 2, S, C>::run(e);
        Dft<R / 2, S, C>::run(o);
        dft_combine<R, S, 0>(x, e, o);
    }
};
template <int S, class C> struct Dft<1, S, C> {
    static __device__ __forceinline__ void run(C*) {}
};
template <int S, class C> struct Dft<2, S, C> {
    static __device__ __forceinline__ void run(C* x) {
        const C a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

// --------------------------------------------------------- exact phase
// Per-node (or per-linear-step) constants.  The dispersion phase
// beta(w_k, z) = w^2/2 I2 + w^3/6 I3 with w = 2 pi k'/T is, in turns,
//   theta = k'^2 a + k'^3 b,  a = pi I2 / T^2,  b = 2 pi^2 I3 / (3 T^3).
// The host stores a mod 1 and b mod 1 as 128-bit binary fractions (exact
// for the FP64 values of a and b); the device reduces theta mod 1 exactly in
// 64-bit integer arithmetic, so no FP64 arithmetic and no large-argument
// range reduction is needed however large beta grows.
struct NodeC {
    unsigned long long a_hi, a_lo, b_hi, b_lo;
    double pre;  // MPA: exp(int_{z0}^{z_j} G) = exp(-gamma (z_j - z0)); SS: linear-step gain
    double post; // MPA: sigma(z_j) dz / pre (weight of V_j in Eq. (6))
};

// frac(k'^2 a + k'^3 b) as an unsigned Q0.64 number of turns (within 2 ulp).
// frac(k'^3 b) = frac(k' frac(k'^2 b)) since k'^3 b - k' frac(k'^2 b) is an
// integer multiple of k'.
__device__ __forceinline__ unsigned long long phase_q64(long long kp, const NodeC& c) {
    const unsigned long long ak = (unsigned long long)(kp < 0 ? -kp : kp);
    const unsigned long long u = ak * ak;  // < 2^50 for N <= 2^25
    const unsigned long long ta = u * c.a_hi + __umul64hi(u, c.a_lo);
    const unsigned long long f_lo = u * c.b_lo;
    const unsigned long long f_hi = u * c.b_hi + __umul64hi(u, c.b_lo);
    unsigned long long tb = ak * f_hi + __umul64hi(ak, f_lo);
    if (kp < 0) tb = 0ull - tb;  // odd power of k'
    return ta + tb;
}

// exp(2 pi i theta) for theta a Q0.64 fraction of a turn: reinterpret as a
// signed fraction in [-1/2, 1/2) and evaluate sin/cos of pi * (2 theta).
template <typename T> __device__ __forceinline__ cx<T> expi_turns(unsigned long long th);
template <> __device__ __forceinline__ float2 expi_turns<float>(unsigned long long th) {
    const float x = __ll2float_rn((long long)th) * 1.0842021724855044e-19f;  // 2^-63
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, s);
}
template <> __device__ __forceinline__ double2 expi_turns<double>(unsigned long long th) {
    const double x = __ll2double_rn((long long)th) * 1.0842021724855044e-19;  // 2^-63
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(c, s);
}

// exp(2 pi i theta) for a Q0.64 turn fraction in FP32 without tables:
// split theta into the nearest quarter turn q and a residual angle
// x = 2 pi (theta - q/4), |x| <= pi/4, evaluate cos x and sin x by their
// Taylor series through x^8 and x^9 (truncation below 2.5e-8 and 1.8e-9),
// and rotate by i^q.
__device__ __forceinline__ float2 expi_turns_poly(unsigned long long th) {
    const unsigned long long q = (th + (1ull << 61)) >> 62;  // 0..3 (the sum wraps at 2^64)
    // residual in units of 2^-32 turn (|d| <= 2^29; the dropped bits are < 2^-32 turn)
    const int d = (int)((long long)(th - (q << 62)) >> 32);
    const float x = __int2float_rn(d) * 1.4629180792671596e-09f;  // 2 pi 2^-32
    const float x2 = x * x;
#if MPA_F32X2 && MPA_F32X2_POLY
    // the cos and sin series side by side in the two lanes of packed FMAs
    const float2 xx = make_float2(x2, x2);
    float2 p = fma2(xx, make_float2(2.4801587e-05f, 2.7557319e-06f), make_float2(-1.3888889e-03f, -1.9841270e-04f));
    p = fma2(p, xx, make_float2(4.1666668e-02f, 8.3333338e-03f));  // 1/4!, 1/5!
    p = fma2(p, xx, make_float2(-0.5f, -0.16666667f));
    const float c = fmaf(p.x, x2, 1.0f);
    const float sn = fmaf(p.y * x2, x, x);
#else
    float c = fmaf(x2, 2.4801587e-05f, -1.3888889e-03f);  // 1/8!, -1/6!
    c = fmaf(c, x2, 4.1666668e-02f);                     // 1/4!
    c = fmaf(c, x2, -0.5f);
    c = fmaf(c, x2, 1.0f);
    float sn = fmaf(x2, 2.7557319e-06f, -1.9841270e-04f);  // 1/9!, -1/7!
    sn = fmaf(sn, x2, 8.3333338e-03f);                     // 1/5!
    sn = fmaf(sn, x2, -0.16666667f);
    sn = fmaf(sn * x2, x, x);
#endif
    // multiply by i^q without branches: odd q swaps (c, s) -> (-s, c), q & 2 negates
    const bool odd = (q & 1) != 0;
    const float a = odd ? -sn : c, b = odd ? c : sn;
    const unsigned neg = (unsigned)(q & 2) << 30;
    return make_float2(__uint_as_float(__float_as_uint(a) ^ neg), __uint_as_float(__float_as_uint(b) ^ neg));
}

// (sin, cos) of a Kerr phase phi = sigma |A|^2 dz of the split-step.  These
// phases are small (about 1e-3 rad on the benchmark links), so for
// |phi| <= 1/16 the Taylor series of cos and sin are used: through phi^8 and
// phi^9 in FP64 (the first dropped terms are below 2.6e-19 and 2.3e-20
// relative) and through phi^4 and phi^5 in FP32 (below 8.3e-11 and 1.2e-11);
// larger phases take the library's sincos.  The FP64 series costs ten
// multiply-adds instead of a full-range evaluation on a GPU whose FP64
// rate is a small fraction of its FP32 rate.
__device__ __forceinline__ void sincos_kerr(double phi, double* s, double* c) {
    if (fabs(phi) <= 0.0625) {
        const double p2 = phi * phi;
        double cc = fma(p2, 1.0 / 40320.0, -1.0 / 720.0);
        cc = fma(cc, p2, 1.0 / 24.0);
        cc = fma(cc, p2, -0.5);
        *c = fma(cc, p2, 1.0);
        double ss = fma(p2, 1.0 / 362880.0, -1.0 / 5040.0);
        ss = fma(ss, p2, 1.0 / 120.0);
        ss = fma(ss, p2, -1.0 / 6.0);
        *s = fma(ss * p2, phi, phi);
    } else {
        sincos(phi, s, c);
    }
}
__device__ __forceinline__ void sincos_kerr(float phi, float* s, float* c) {
    if (fabsf(phi) <= 0.0625f) {
        const float p2 = phi * phi;
        *c = fmaf(fmaf(p2, 1.0f / 24.0f, -0.5f), p2, 1.0f);
        *s = fmaf(fmaf(p2, 1.0f / 120.0f, -1.0f / 6.0f) * p2, phi, phi);
    } else {
        sincosf(phi, s, c);
    }
}

// Exact phases theta(k'_0 + s D), s = -R/2 .. R/2-1, produced in s order
// by finite differences in Q0.64 arithmetic: theta is a cubic in s, so
// after four direct evaluations every further value costs three 64-bit
// additions (each direct value is within 2 ulp of 2^-64; over 32 values
// the cubic extrapolation keeps the error below 2^-48 turns).
struct PhaseRun {
    unsigned long long t0, t1, t2, t3, d1, d2, d3;
    int n;
    __device__ __forceinline__ PhaseRun(long long k_first, long long D, const NodeC& c) : n(0) {
        t0 = phase_q64(k_first, c);
        t1 = phase_q64(k_first + D, c);
        t2 = phase_q64(k_first + 2 * D, c);
        t3 = phase_q64(k_first + 3 * D, c);
        d1 = t3 - t2;
        d2 = t3 - 2 * t2 + t1;
        d3 = t3 - 3 * t2 + 3 * t1 - t0;
    }
    // value number n (n = 0, 1, 2, ...) of the progression
    __device__ __forceinline__ unsigned long long next() {
        const int m = n++;
        if (m == 0) return t0;
        if (m == 1) return t1;
        if (m == 2) return t2;
        if (m == 3) return t3;
        d2 += d3;
        d1 += d2;
        t3 += d1;
        return t3;
    }
};

// Phases of the R elements k'_s = k'_0 + s D, s = -R/2 .. R/2-1 of one
// butterfly by exact finite differences in Q0.64 arithmetic: theta is a
// cubic in s, so after four direct evaluations every further value costs
// three 64-bit additions (the direct values are within 2 ulp of 2^-64, so
// over 32 values the error stays below 2^-48 turns).  th[r] receives the phase
// of element r, where s = r for r < R/2 and s = r - R for r >= R/2.
template <int R>
__device__ __forceinline__ void phase_run(long long k0, long long D, const NodeC& c, unsigned long long (&th)[R]) {
    static_assert(R >= 4, "finite differences need four points");
    const long long ks = k0 - (long long)(R / 2) * D;
    unsigned long long t0 = phase_q64(ks, c), t1 = phase_q64(ks + D, c), t2 = phase_q64(ks + 2 * D, c),
                       t3 = phase_q64(ks + 3 * D, c);
    unsigned long long d1 = t3 - t2, d2 = t3 - 2 * t2 + t1, d3 = t3 - 3 * t2 + 3 * t1 - t0;
    th[R / 2] = t0;
    th[R / 2 + 1] = t1;
    th[R / 2 + 2] = t2;
    th[R / 2 + 3] = t3;
    unsigned long long t = t3;
#pragma unroll
    for (int s = -R / 2 + 4; s < R / 2; ++s) {
        d2 += d3;
        d1 += d2;
        t += d1;
        th[(s + R) % R] = t;
    }
}

// exp(2 pi i e / n) for an integer e (|e| small enough to be exact in T
// after reduction to [-n/2, n/2)), n a power of two given by log2.
template <typename T> __device__ __forceinline__ cx<T> expi_ratio(long long e, int log2n) {
    const long long n = 1ll << log2n;
    e &= (n - 1);
    if (e >= (n >> 1)) e -= n;
    T s, c;
    if constexpr (sizeof(T) == 4) {
        // |e| <= 2^24 here: a 32-bit conversion (a 64-bit one runs on the
        // FP64 pipe) and an exact scaling by the power of two 2^(1 - log2n)
        const float x = (float)(int)e * __int_as_float((128 - log2n) << 23);
        sincospif(x, &s, &c);
    } else {
        const double x = (double)e * 2.0 / (double)n;  // exact: |e| <= 2^52
        sincospi(x, &s, &c);
    }
    return mkc(c, s);
}

// ------------------------------------------------- thread groups
// A transform runs on the whole block (GRP = 0: threadIdx.x, __syncthreads)
// or on one of several NT-thread groups of the block (GRP = 1: the thread's
// index within its group, and named barrier 1 + group over the group's NT
// threads, so groups never wait on one another).
template <int GRP, int NT> __device__ __forceinline__ int gtid() {
    if constexpr (GRP == 0) return threadIdx.x;
    else return threadIdx.x & (NT - 1);
}
template <int GRP, int NT> __device__ __forceinline__ void gsync() {
    if constexpr (GRP == 0) {
        __syncthreads();
    } else {
        static_assert((NT & (NT - 1)) == 0 && NT % 32 == 0, "groups of whole warps, a power of two");
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / NT)), "n"(NT) : "memory");
    }
}

// ------------------------------------------------- shared-memory Stockham
// Padding of the shared-memory tile: one extra element per 2^PSH elements
// keeps every pass free of bank conflicts (PSH = log2 of the largest radix).
template <int PSH> __host__ __device__ __forceinline__ int phys(int i) { return i + (i >> PSH); }

// Tile layouts of G independent transforms of length L:
//   COL: element (l, g) at l*G + g  (a tile of G columns of an N2 x N1 matrix)
//   ROW: element (l, g) at g*L + l  (G contiguous rows)
enum { LAYOUT_COL = 0, LAYOUT_ROW = 1 };

template <int LAYOUT, int L, int G> __host__ __device__ __forceinline__ int eidx(int l, int g) {
    return LAYOUT == LAYOUT_COL ? l * G + g : g * L + l;
}

// The padded slot phys(eidx(l, g)) for l = lb + c written as base(lb, g) +
// off(c): with c a compile-time constant of an unrolled loop, off(c) folds
// into the shared-memory instruction's immediate offset, so each element
// costs no integer work.  The padding term i >> PSH is
//   COL, G >= 2^PSH: l (G >> PSH) + (g >> PSH)        (no condition)
//   COL, G <  2^PSH: l >> SH, SH = PSH - log2 G       (as g < G)
//   ROW, L >= 2^PSH: g (L >> PSH) + (l >> PSH)        (SH = PSH)
//   ROW, L <  2^PSH: g >> (PSH - log2 L)              (no condition)
// and the split is exact when (lb + c) >> SH = (lb >> SH) + (c >> SH) for
// every c the caller adds (strided() states the cases the passes use).
// Sites of the column layout that use the split form: bits 0-3 for
// transforms with the small radix last (SF false), bits 4-7 for those with
// it first (bit 0: first-pass scatter, 1: middle-pass reads, 2: middle-pass
// writes, 3: last-pass gather); the row layout uses it wherever it is
// exact.  Measured on the 2^20 link (split 2^12 x 2^8): the split row
// layout takes the row pass from 3223 to 3316 GB/s.  In the column layout
// it cuts instructions in both directions, but the forward column pass
// (radix 8 then 32, a 32-element gather per thread) fell from 3816 to
// 3417 GB/s while the inverse one (32 then 8) rose from 2906 to 2992 GB/s.
#ifndef MPA_SLOT_COL
#define MPA_SLOT_COL 0x0F
#endif
template <int LAYOUT, bool SF, int SITE> __host__ __device__ constexpr bool slot_site_on() {
    return LAYOUT != LAYOUT_COL || ((MPA_SLOT_COL >> (SITE + (SF ? 4 : 0))) & 1) != 0;
}

template <int LAYOUT, int L, int G, int PSH> struct Slot {
    __host__ __device__ static constexpr int lg(int x) { return x <= 1 ? 0 : 1 + lg(x / 2); }
    static constexpr int P2 = 1 << PSH;
    static constexpr bool COL = LAYOUT == LAYOUT_COL;
    // l enters through a shift by SH (else the split needs no condition)
    static constexpr bool LDEP = COL ? (G < P2) : (L >= P2);
    static constexpr int SH = COL ? (G < P2 ? PSH - lg(G) : 0) : (L >= P2 ? PSH : 0);
    static __host__ __device__ __forceinline__ int base(int lb, int g) {
        if constexpr (COL) {
            if constexpr (G >= P2) return lb * (G + (G >> PSH)) + g + (g >> PSH);
            else return lb * G + g + (lb >> SH);
        } else {
            if constexpr (L >= P2) return g * (L + (L >> PSH)) + lb + (lb >> PSH);
            else return g * L + (g >> (PSH - lg(L))) + lb;
        }
    }
    static __host__ __device__ constexpr int off(int c) {
        return COL ? (G >= P2 ? c * (G + (G >> PSH)) : c * G + (c >> SH)) : (L >= P2 ? c + (c >> PSH) : c);
    }
    // lb + r STRIDE with 0 <= lb < STRIDE, r < R: the shift splits if STRIDE
    // is a multiple of 2^SH or the whole range R STRIDE fits below 2^SH
    template <int STRIDE, int R> __host__ __device__ static constexpr bool strided() {
        return !LDEP || STRIDE % (1 << SH) == 0 || STRIDE * R <= (1 << SH);
    }
};

// Two-level table of W_L^e = exp(2 pi i e/L): hi[e >> SH] * lo[e & (2^SH-1)].
template <int L> struct TwDims {
    static constexpr int logL = (L >= 16384) ? 14 : (L >= 8192) ? 13 : (L >= 4096) ? 12 : (L >= 2048) ? 11
                              : (L >= 1024) ? 10 : (L >= 512) ? 9 : (L >= 256) ? 8 : (L >= 128) ? 7
                              : (L >= 64) ? 6 : (L >= 32) ? 5 : (L >= 16) ? 4 : (L >= 8) ? 3 : (L >= 4) ? 2 : 1;
    static constexpr int SH = (logL + 1) / 2;
    static constexpr int NLO = 1 << SH;
    static constexpr int NHI = L >> SH;
};

// Slot of entry e of the low twiddle table.  A row-pass warp looks up
// e = s j for 32 consecutive j and a power of two s; 8-byte entries sit in 16
// bank pairs, so in natural order the stride s = 4, 8, 16 lookups would
// collide 4- to 8-fold.  XOR-ing the entry's 16-block index into its low
// four bits spreads every such stride over distinct bank pairs.
template <int NLO> __device__ __forceinline__ int tw_lo_slot(int e) {
    if constexpr (NLO >= 32) return e ^ ((e >> 4) & 15);
    else return e;
}

template <typename T, int L> __device__ __forceinline__ void tw_init(cx<T>* hi, cx<T>* lo, int tid, int nt) {
    typedef TwDims<L> D;
    for (int i = tid; i < D::NLO + D::NHI; i += nt) {
        if (i < D::NLO) lo[tw_lo_slot<D::NLO>(i)] = expi_ratio<T>(i, D::logL);
        else hi[i - D::NLO] = expi_ratio<T>((long long)(i - D::NLO) << D::SH, D::logL);
    }
}

template <typename T, int L> __device__ __forceinline__ cx<T> tw_get(const cx<T>* hi, const cx<T>* lo, int e) {
    typedef TwDims<L> D;
    if constexpr (D::NHI == 1) return lo[tw_lo_slot<D::NLO>(e)];
    else return cmul(hi[e >> D::SH], lo[tw_lo_slot<D::NLO>(e & (D::NLO - 1))]);
}

// v[r] *= W_L^{S r e1} for r = 1..R-1 (R <= 32): table lookups of
// w1, w2, w4 (combined into w1..w7) and w8, w16 (w24 = w8 w16), then
// w_r = w_{r mod 8} w_{8 floor(r/8)}, at most three products deep.
template <typename T, int L, int R, int S>
__device__ __forceinline__ void twiddle_row(cx<T>* v, int e1, const cx<T>* hi, const cx<T>* lo) {
    typedef cx<T> C;
    C w[8];
    w[1] = tw_get<T, L>(hi, lo, e1);
    if constexpr (R > 2) w[2] = tw_get<T, L>(hi, lo, 2 * e1);
    if constexpr (R > 2) w[3] = cmul(w[1], w[2]);
    if constexpr (R > 4) {
        w[4] = tw_get<T, L>(hi, lo, 4 * e1);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
    }
    C u[4];
    if constexpr (R > 8) u[1] = tw_get<T, L>(hi, lo, 8 * e1);
    if constexpr (R > 16) {
        u[2] = tw_get<T, L>(hi, lo, 16 * e1);
        u[3] = cmul(u[1], u[2]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const int a = r & 7, b = r >> 3;
        C t;
        if (b == 0) t = w[a];
        else if (a == 0) t = u[b];
        else t = cmul(w[a], u[b]);
        v[r] = mul_dir<S>(v[r], t);
    }
}

// One radix-R Stockham pass over the tile (in place, barrier-separated
// read and write phases).  Butterfly j of transform g reads elements
// j + r L/R, applies W_{NS R}^{S r (j mod NS)}, does the R-point DFT and
// writes to (j - j mod NS) R + j mod NS + r NS.
template <typename T, int L, int G, int NT, int R, int NS, int S, int LAYOUT, int PSH, bool SF, int GRP = 0>
__device__ __forceinline__ void stockham_pass(cx<T>* s, const cx<T>* hi, const cx<T>* lo) {
    typedef cx<T> C;
    constexpr int NB = (L / R) * G;
    static_assert(NB % NT == 0, "butterflies must divide among threads");
    constexpr int Q = NB / NT;
    C v[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = gtid<GRP, NT>() + q * NT;
        const int j = LAYOUT == LAYOUT_COL ? b / G : b % (L / R);
        const int g = LAYOUT == LAYOUT_COL ? b % G : b / (L / R);
        typedef Slot<LAYOUT, L, G, PSH> SL;
        if constexpr (slot_site_on<LAYOUT, SF, 1>() && SL::template strided<L / R, R>()) {
            const C* sb = s + SL::base(j, g);
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = sb[SL::off(r * (L / R))];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = s[phys<PSH>(eidx<LAYOUT, L, G>(j + r * (L / R), g))];
        }
        if constexpr (NS > 1) twiddle_row<T, L, R, S>(v[q], (j & (NS - 1)) * (L / (NS * R)), hi, lo);
        Dft<R, S, C>::run(v[q]);
    }
    gsync<GRP, NT>();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = gtid<GRP, NT>() + q * NT;
        const int j = LAYOUT == LAYOUT_COL ? b / G : b % (L / R);
        const int g = LAYOUT == LAYOUT_COL ? b % G : b / (L / R);
        const int k = j & (NS - 1);
        const int dst = (j - k) * R + k;
        typedef Slot<LAYOUT, L, G, PSH> SL;
        // dst = m NS R + k (k < NS): the offsets r NS stay below NS R
        if constexpr (slot_site_on<LAYOUT, SF, 2>() && SL::template strided<NS, R>()) {
            C* sb = s + SL::base(dst, g);
#pragma unroll
            for (int r = 0; r < R; ++r) sb[SL::off(r * NS)] = v[q][r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) s[phys<PSH>(eidx<LAYOUT, L, G>(dst + r * NS, g))] = v[q][r];
        }
    }
    gsync<GRP, NT>();
}

// Pass schedule of a length-L transform with radices RMAX and one smaller
// radix 2^b when log2 L is not a multiple of log2 RMAX.  SMALL_FIRST puts
// the small radix first (the transform then ends with an RMAX pass), else
// last.  Two transforms meet in registers when the last radix of the first
// equals the first radix of the second: the last pass leaves element
// j + r L/R of butterfly j in v[r], which is exactly what a first pass of
// the same radix reads.
template <int L, int RMAX> struct Sched {
    __host__ __device__ static constexpr int lg(int x) { return x <= 1 ? 0 : 1 + lg(x / 2); }
    static constexpr int LOGL = lg(L), LOGR = lg(RMAX);
    static constexpr int NFULL = LOGL / LOGR;
    static constexpr int SMALL = 1 << (LOGL % LOGR);  // 1 if none
    static constexpr int NP = NFULL + (SMALL > 1 ? 1 : 0);
    template <bool SF> __host__ __device__ static constexpr int radix(int p) {
        return SMALL == 1 ? RMAX : SF ? (p == 0 ? SMALL : RMAX) : (p == NP - 1 ? SMALL : RMAX);
    }
    template <bool SF> __host__ __device__ static constexpr int ns(int p) { return p == 0 ? 1 : ns<SF>(p - 1) * radix<SF>(p - 1); }
};

template <typename T, int L, int G, int NT, int RMAX, int S, int LAYOUT, int PSH, bool SF, int P, int NP, int GRP = 0>
__device__ __forceinline__ void mid_passes(cx<T>* s, const cx<T>* hi, const cx<T>* lo) {
    if constexpr (P < NP - 1) {
        typedef Sched<L, RMAX> SC;
        stockham_pass<T, L, G, NT, SC::template radix<SF>(P), SC::template ns<SF>(P), S, LAYOUT, PSH, SF, GRP>(s, hi,
                                                                                                              lo);
        mid_passes<T, L, G, NT, RMAX, S, LAYOUT, PSH, SF, P + 1, NP, GRP>(s, hi, lo);
    }
}

// Butterfly b of a radix-R pass -> (j, g).
template <int LAYOUT, int L, int G, int R> __host__ __device__ __forceinline__ void bmap(int b, int& j, int& g) {
    if constexpr (LAYOUT == LAYOUT_COL) {
        j = b / G;
        g = b % G;
    } else {
        j = b % (L / R);
        g = b / (L / R);
    }
}

// A whole transform with register endpoints.  vin[q][r] holds input element
// j + r L/R0 of butterfly b = tid + q NT (R0 = first radix), vout[q][r]
// receives output element j + r L/RL (RL = last radix).  Shared memory is
// used by the middle passes only; the transform ends with a barrier so the
// caller may reuse `s`.  GRP as for gtid/gsync.
template <typename T, int L, int G, int NT, int RMAX, int S, int LAYOUT, int PSH, bool SF, int GRP = 0> struct Xform {
    typedef Sched<L, RMAX> SC;
    typedef cx<T> C;
    static constexpr int NP = SC::NP;
    static constexpr int R0 = SC::template radix<SF>(0);
    static constexpr int RL = SC::template radix<SF>(NP - 1);
    static constexpr int Q0 = (L / R0) * G / NT;
    static constexpr int QL = (L / RL) * G / NT;
    static_assert((L / R0) * G % NT == 0 && (L / RL) * G % NT == 0, "butterflies must divide among threads");

    struct NoHook {
        __device__ __forceinline__ void operator()() const {}
    };
    static __device__ __forceinline__ void run(C (&vin)[Q0][R0], C (&vout)[QL][RL], C* s, const C* hi, const C* lo) {
        run(vin, vout, s, hi, lo, NoHook());
    }
    // hook() runs once the first pass has left the registers for shared
    // memory (after its barrier; at the start for a single-pass transform),
    // where the caller's own work needs the fewest registers.
    template <class Hook>
    static __device__ __forceinline__ void run(C (&vin)[Q0][R0], C (&vout)[QL][RL], C* s, const C* hi, const C* lo,
                                               Hook&& hook) {
        if constexpr (NP == 1) {
            hook();
#pragma unroll
            for (int q = 0; q < Q0; ++q) {
                Dft<R0, S, C>::run(vin[q]);
#pragma unroll
                for (int r = 0; r < R0; ++r) vout[q][r] = vin[q][r];
            }
        } else {
            // first pass: DFT of the register inputs (NS = 1), scatter to j R0 + r
#pragma unroll
            for (int q = 0; q < Q0; ++q) {
                int j, g;
                bmap<LAYOUT, L, G, R0>(gtid<GRP, NT>() + q * NT, j, g);
                Dft<R0, S, C>::run(vin[q]);
                // j R0 + r, r < R0: the shift always splits (j R0 is a multiple
                // of 2^SH, or R0 divides 2^SH and r < R0 adds no carry)
                typedef Slot<LAYOUT, L, G, PSH> SL;
                if constexpr (slot_site_on<LAYOUT, SF, 0>()) {
                    C* sb = s + SL::base(j * R0, g);
#pragma unroll
                    for (int r = 0; r < R0; ++r) sb[SL::off(r)] = vin[q][r];
                } else {
#pragma unroll
                    for (int r = 0; r < R0; ++r) s[phys<PSH>(eidx<LAYOUT, L, G>(j * R0 + r, g))] = vin[q][r];
                }
            }
            gsync<GRP, NT>();
            hook();
            mid_passes<T, L, G, NT, RMAX, S, LAYOUT, PSH, SF, 1, NP, GRP>(s, hi, lo);
            // last pass (NS = L/RL, so k = j): gather j + r L/RL, twiddle W_L^{S r j}, DFT
#pragma unroll
            for (int q = 0; q < QL; ++q) {
                int j, g;
                bmap<LAYOUT, L, G, RL>(gtid<GRP, NT>() + q * NT, j, g);
                typedef Slot<LAYOUT, L, G, PSH> SL;
                if constexpr (slot_site_on<LAYOUT, SF, 3>() && SL::template strided<L / RL, RL>()) {
                    const C* sb = s + SL::base(j, g);
#pragma unroll
                    for (int r = 0; r < RL; ++r) vout[q][r] = sb[SL::off(r * (L / RL))];
                } else {
#pragma unroll
                    for (int r = 0; r < RL; ++r) vout[q][r] = s[phys<PSH>(eidx<LAYOUT, L, G>(j + r * (L / RL), g))];
                }
                twiddle_row<T, L, RL, S>(vout[q], j, hi, lo);
                Dft<RL, S, C>::run(vout[q]);
            }
            gsync<GRP, NT>();
        }
    }
};

// Precision-dependent tiling: elements per thread E, largest radix, the
// padding shift, the minimum column-tile width (64-byte row segments) and
// the target tile size in elements.
// KIND 0 = column pass, 1 = row pass (tuned separately).
#ifndef MPA_KC_E
#define MPA_KC_E 32
#endif
#ifndef MPA_KC_TE
#define MPA_KC_TE 8192
#endif
#ifndef MPA_KR_E
#define MPA_KR_E 32
#endif
#ifndef MPA_KR_TE
#define MPA_KR_TE 8192
#endif
#ifndef MPA_KCW_E
#define MPA_KCW_E 16
#endif
// KIND 2 = wavefront column pass.
template <typename T, int KIND = 0> struct Tiling;
#ifndef MPA_RMAX32
#define MPA_RMAX32 32
#endif
template <int KIND> struct Tiling<float, KIND> {
    // radix-32 passes (one smem exchange for a 1024-point transform) where a
    // thread holds 32 elements; the wavefront pass (16 per thread) uses 16
    static constexpr int E = KIND == 0 ? MPA_KC_E : KIND == 1 ? MPA_KR_E : MPA_KCW_E;
    static constexpr int RMAX = E >= 32 ? MPA_RMAX32 : 16, PSH = RMAX == 32 ? 5 : 4, CMIN = 8;
    static constexpr int TE = KIND == 1 ? MPA_KR_TE : MPA_KC_TE;
};
template <int KIND> struct Tiling<double, KIND> {
    static constexpr int E = 16, RMAX = 8, PSH = 3, CMIN = 4, TE = 4096;
};

}  // namespace mpa
