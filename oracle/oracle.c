/*
 * FP64 CPU oracle: plain, slow, step-by-step restatement of the paper's
 * method.  TEST INFRASTRUCTURE ONLY (see oracle.h): nothing on the product
 * path links or calls this file.
 *
 * Paper passages followed:
 *   Eq. (1)            the NLSE, G(z) = -gamma + g(z) + (e^{z_a gamma}-1) sum delta(z - z_k),
 *                      g(z) a distributed gain that is constant on each segment
 *   text after Eq. (1) Fourier transform with exp(+i omega t); interaction
 *                      picture A_hat = psi_hat exp(i beta + int G); beta(omega, z)
 *   Eq. (2)            integral equation for psi_hat
 *   MPA steps 1-7      Picard iteration over one interval [z0, z0+L]
 *   Eq. (6)            trapezoidal discretisation of the iteration
 *   Eq. (4)            composite (Strang) split-step
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#define ORACLE_MAX_THREADS() omp_get_max_threads()
#else
#define ORACLE_MAX_THREADS() 1
#endif

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------ FFT */

static int is_pow2(long n) { return n >= 2 && (n & (n - 1)) == 0; }

/* Iterative radix-2 Cooley-Tukey, decimation in time: bit-reverse the
 * input, then log2(N) butterfly stages.  Twiddles exp(sign 2 pi i m/N) are
 * evaluated directly with libm for every m (no recurrences). */
static int fft_c(cplx* x, long N, int sign) {
    if (!is_pow2(N)) return 1;
    for (long i = 1, j = 0; i < N; i++) {
        long bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    long half_n = N / 2;
    cplx* tw = (cplx*)malloc(sizeof(cplx) * (size_t)half_n);
    if (!tw) return 3;
    for (long m = 0; m < half_n; m++) {
        double a = TWO_PI * (double)m / (double)N;
        tw[m] = cos(a) + I * (sign > 0 ? sin(a) : -sin(a));
    }
    for (long len = 2; len <= N; len <<= 1) {
        long half = len / 2, step = N / len;
        for (long i = 0; i < N; i += len) {
            for (long m = 0; m < half; m++) {
                cplx w = tw[m * step];
                cplx u = x[i + m];
                cplx v = x[i + m + half] * w;
                x[i + m] = u + v;
                x[i + m + half] = u - v;
            }
        }
    }
    free(tw);
    if (sign < 0) {
        double s = 1.0 / (double)N;
        for (long i = 0; i < N; i++) x[i] *= s;
    }
    return 0;
}

int oracle_fft(double* x, long N, int sign) { return fft_c((cplx*)x, N, sign); }

/* ------------------------------------------------------------ fiber map */

/* columns of a segment row: length, beta2, beta3, sigma, distributed gain */
#define NCOL 5

typedef struct {
    const double* rows; /* n_seg x {length, beta2, beta3, sigma, gain} */
    int n_seg;
    double gamma, z_a;
    int n_periods;
    double period;
} fmap;

static fmap make_map(const double* rows, int n_seg, double gamma, double z_a, int n_periods) {
    fmap m = {rows, n_seg, gamma, z_a, n_periods, 0.0};
    for (int s = 0; s < n_seg; s++) m.period += rows[NCOL * s];
    return m;
}

/* int_za^zb of coefficient column col (1 = beta2, 2 = beta3, 3 = sigma,
 * 4 = distributed gain):
 * sum over every segment copy of coefficient x overlap length. */
static double integrate(const fmap* m, double za, double zb, int col) {
    if (zb <= za) return 0.0;
    double acc = 0.0;
    long p0 = (long)floor(za / m->period) - 1, p1 = (long)floor(zb / m->period) + 1;
    for (long p = p0; p <= p1; p++) {
        double off = (double)p * m->period;
        for (int s = 0; s < m->n_seg; s++) {
            double a = off, b = off + m->rows[NCOL * s];
            off = b;
            double lo = a > za ? a : za, hi = b < zb ? b : zb;
            if (hi > lo) acc += m->rows[NCOL * s + col] * (hi - lo);
        }
    }
    return acc;
}

/* Coefficient value just left (side < 0) or right (side > 0) of z. */
static double coef_side(const fmap* m, double z, int col, int side) {
    double eps = 1e-9 * m->period;
    double zz = z + (side > 0 ? eps : -eps);
    double u = zz - floor(zz / m->period) * m->period;
    double off = 0.0;
    for (int s = 0; s < m->n_seg; s++) {
        double b = off + m->rows[NCOL * s];
        if (u < b || s == m->n_seg - 1) return m->rows[NCOL * s + col];
        off = b;
    }
    return m->rows[NCOL * (m->n_seg - 1) + col];
}

/* Number of amplifiers z_k = k z_a (k >= 1) with za < z_k <= zb. */
static long n_amps(const fmap* m, double za, double zb) {
    if (m->z_a <= 0.0) return 0;
    double tol = 1e-9 * m->z_a;
    long ka = (long)floor((za + tol) / m->z_a), kb = (long)floor((zb + tol) / m->z_a);
    if (ka < 0) ka = 0;
    return kb > ka ? kb - ka : 0;
}

/* 1 if an amplifier z_k = k z_a (k >= 1) lies strictly inside (za, zb):
 * more than n_amps' tolerance away from both ends.  The MPA applies the
 * lumped gain only at an interval end (step 7), so such an interval is
 * rejected. */
static int amp_inside(const fmap* m, double za, double zb) {
    if (m->z_a <= 0.0) return 0;
    double tol = 1e-9 * m->z_a;
    long first = (long)floor((za + tol) / m->z_a) + 1; /* smallest k with k z_a > za + tol */
    long last = (long)ceil((zb - tol) / m->z_a) - 1;   /* largest k with k z_a < zb - tol */
    if (first < 1) first = 1;
    return last >= first;
}

/* int_za^zb G without the lumped amplifiers: -gamma (zb - za) plus the
 * distributed gain of the segments (G of Eq. (1) between the z_k). */
static double int_G(const fmap* m, double za, double zb) {
    return -m->gamma * (zb - za) + integrate(m, za, zb, 4);
}

static double omega_of(long k, long N, double T) {
    long kp = k < N / 2 ? k : k - N;
    return TWO_PI * (double)kp / T;
}

/* beta(omega, za, zb) of the text after Eq. (2), evaluated in FP64. */
static double beta_of(double w, double I2, double I3) { return 0.5 * w * w * I2 + w * w * w * I3 / 6.0; }

/* Exact linear flow over [za, zb] on a spectrum (the sigma = 0 solution of
 * Eq. (2), continued across amplifiers). */
static void linear_flow(const fmap* m, cplx* X, long N, double T, double za, double zb) {
    double I2 = integrate(m, za, zb, 1), I3 = integrate(m, za, zb, 2);
    double g = exp(int_G(m, za, zb) + (double)n_amps(m, za, zb) * m->z_a * m->gamma);
    for (long k = 0; k < N; k++) {
        double b = beta_of(omega_of(k, N, T), I2, I3);
        X[k] *= g * (cos(b) + I * sin(b));
    }
}

static int check_span(const fmap* m, double z_from, double z_to) {
    if (!(z_to >= z_from) || z_from < -1e-12) return 2;
    if (z_to > m->period * m->n_periods * (1.0 + 1e-12) + 1e-9) return 2;
    return 0;
}

/* ----------------------------------------------------------------- MPA */

/* One interval of the MPA (steps 1-6 of the algorithm, Eq. (6)): returns
 * psi^{(n_tot)} at node M.  psi0 is the spectrum A_hat(z0) in natural order. */
static int mpa_interval(const fmap* m, long N, double T, double z0, double L, int M, int n_tot,
                        const cplx* psi0, cplx* psiM, int n_threads) {
    double dz = L / (double)M;
    size_t nn = (size_t)(M + 1) * (size_t)N;
    cplx* psi = (cplx*)malloc(sizeof(cplx) * nn);
    cplx* V = (cplx*)malloc(sizeof(cplx) * nn);
    double* I2 = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* I3 = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* sig = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* loss = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    if (!psi || !V || !I2 || !I3 || !sig || !loss) {
        free(psi); free(V); free(I2); free(I3); free(sig); free(loss);
        return 3;
    }
    /* per-node quantities: z_j = z0 + j dz, beta relative to z0, the loss
     * factor exp(int_{z0}^{z_j} G) (loss and distributed gain) and sigma(z_j)
     * (average of the one-sided values where a segment boundary falls on an
     * interior node, the inner one-sided value at the interval ends). */
    for (int j = 0; j <= M; j++) {
        double zj = z0 + dz * (double)j;
        I2[j] = integrate(m, z0, zj, 1);
        I3[j] = integrate(m, z0, zj, 2);
        loss[j] = exp(int_G(m, z0, zj));
        if (j == 0) sig[j] = coef_side(m, zj, 3, +1);
        else if (j == M) sig[j] = coef_side(m, zj, 3, -1);
        else sig[j] = 0.5 * (coef_side(m, zj, 3, -1) + coef_side(m, zj, 3, +1));
    }
    /* step 1: copy psi(z0) to every node */
    for (int j = 0; j <= M; j++) memcpy(psi + (size_t)j * N, psi0, sizeof(cplx) * (size_t)N);

    int err = 0;
    for (int it = 0; it < n_tot; it++) {
        /* steps 2-4 at every node, independently (one node per task) */
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : ORACLE_MAX_THREADS())
        for (int j = 0; j <= M; j++) {
            cplx* a = (cplx*)malloc(sizeof(cplx) * (size_t)N);
            if (!a) { err = 3; continue; }
            const cplx* pj = psi + (size_t)j * N;
            for (long k = 0; k < N; k++) {
                double b = beta_of(omega_of(k, N, T), I2[j], I3[j]);
                a[k] = pj[k] * (cos(b) + I * sin(b)) * loss[j];            /* step 2 */
            }
            fft_c(a, N, -1);                                                 /* step 3 */
            for (long n = 0; n < N; n++) {
                double p = creal(a[n]) * creal(a[n]) + cimag(a[n]) * cimag(a[n]);
                a[n] *= p;                                                   /* |A|^2 A */
            }
            fft_c(a, N, +1);                                                 /* step 4 */
            cplx* vj = V + (size_t)j * N;
            for (long k = 0; k < N; k++) {
                double b = beta_of(omega_of(k, N, T), I2[j], I3[j]);
                /* V_j = sigma(z_j) F[|A_j|^2 A_j] dz exp(-i beta - int G), Eq. (6) */
                vj[k] = sig[j] * dz * a[k] * (cos(b) - I * sin(b)) / loss[j];
            }
            free(a);
        }
        if (err) break;
        /* step 5: trapezoidal rule with every partial integral saved,
         * psi_l = psi_0 + i (V_0/2 + sum_{j=1}^{l-1} V_j + V_l/2), l = 1..M */
        for (long k = 0; k < N; k++) {
            cplx run = 0.5 * V[k];
            for (int l = 1; l <= M; l++) {
                cplx vl = V[(size_t)l * N + k];
                psi[(size_t)l * N + k] = psi0[k] + I * (run + 0.5 * vl);
                run += vl;
            }
        }
        /* step 6: the next iteration starts again at step 2 */
    }
    if (!err) memcpy(psiM, psi + (size_t)M * N, sizeof(cplx) * (size_t)N);
    free(psi); free(V); free(I2); free(I3); free(sig); free(loss);
    return err;
}

int oracle_mpa_interval(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
                        long N, double T, double z0, double L, int M, int n_tot,
                        const double* psi0, double* psiM, int n_threads) {
    if (!is_pow2(N)) return 1;
    if (M < 1 || n_tot < 1 || !(L > 0.0) || !(T > 0.0) || n_seg < 1) return 4;
    fmap m = make_map(seg_rows, n_seg, gamma, z_a, n_periods);
    return mpa_interval(&m, N, T, z0, L, M, n_tot, (const cplx*)psi0, (cplx*)psiM, n_threads);
}

int oracle_mpa(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
               long N, double T, double z_from, double z_to, double L, int M, int n_tot,
               double* field, int n_threads, int* threads_used) {
    if (!is_pow2(N)) return 1;
    if (M < 1 || n_tot < 1 || !(L > 0.0) || !(T > 0.0) || n_seg < 1) return 4;
    fmap m = make_map(seg_rows, n_seg, gamma, z_a, n_periods);
    if (check_span(&m, z_from, z_to)) return 2;
    double cnt = (z_to - z_from) / L;
    long n_int = lround(cnt);
    if (fabs(cnt - (double)n_int) > 1e-9 * (cnt > 1.0 ? cnt : 1.0)) return 2;
    /* amplifiers may only sit at interval ends */
    for (long q = 0; q < n_int; q++) {
        double a = z_from + L * (double)q, b = z_from + L * (double)(q + 1);
        if (amp_inside(&m, a, b)) return 2;
    }
    if (threads_used) {
        *threads_used = n_threads > 0 ? n_threads : ORACLE_MAX_THREADS();
    }
    cplx* X = (cplx*)field;
    cplx* psiM = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    if (!psiM) return 3;
    fft_c(X, N, +1); /* A_hat(z_from) = psi_hat(z0) of the first interval */
    int err = 0;
    for (long q = 0; q < n_int && !err; q++) {
        double z0 = z_from + L * (double)q;
        err = mpa_interval(&m, N, T, z0, L, M, n_tot, X, psiM, n_threads);
        if (err) break;
        /* step 7: A_hat(z0 + L) = psi_M exp(i beta(omega, z0 + L) + int G),
         * then the lumped gain when z0 + L is an amplifier location */
        double I2 = integrate(&m, z0, z0 + L, 1), I3 = integrate(&m, z0, z0 + L, 2);
        double g = exp(int_G(&m, z0, z0 + L) + (double)n_amps(&m, z0, z0 + L) * m.z_a * m.gamma);
        for (long k = 0; k < N; k++) {
            double b = beta_of(omega_of(k, N, T), I2, I3);
            X[k] = psiM[k] * (cos(b) + I * sin(b)) * g;
        }
    }
    free(psiM);
    fft_c(X, N, -1);
    return err;
}

/* ------------------------------------------------------------------ SS */

int oracle_ss(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
              long N, double T, double z_from, double z_to, double dz, double* field) {
    if (!is_pow2(N)) return 1;
    if (!(dz > 0.0) || !(T > 0.0) || n_seg < 1) return 4;
    fmap m = make_map(seg_rows, n_seg, gamma, z_a, n_periods);
    if (check_span(&m, z_from, z_to)) return 2;
    double cnt = (z_to - z_from) / dz;
    long K = lround(cnt);
    if (K < 1 || fabs(cnt - (double)K) > 1e-9 * (cnt > 1.0 ? cnt : 1.0)) return 2;
    cplx* X = (cplx*)field;
    fft_c(X, N, +1);
    /* Eq. (4): exp(iL dz/2) Q^K exp(-iL dz/2), Q = exp(iN dz) exp(iL dz):
     * half linear step, then K nonlinear kicks at the step midpoints
     * z_k + dz/2 separated by full linear steps, and a final half step. */
    double za = z_from, zb = z_from + 0.5 * dz;
    linear_flow(&m, X, N, T, za, zb);
    for (long k = 0; k < K; k++) {
        double zk = z_from + dz * (double)k;
        double s = integrate(&m, zk, zk + dz, 3); /* int sigma over the step */
        fft_c(X, N, -1);
        for (long n = 0; n < N; n++) {
            double p = creal(X[n]) * creal(X[n]) + cimag(X[n]) * cimag(X[n]);
            double ph = s * p;
            X[n] *= cos(ph) + I * sin(ph); /* exp(i sigma |A|^2 dz) A */
        }
        fft_c(X, N, +1);
        za = zb;
        zb = (k == K - 1) ? z_to : zb + dz;
        linear_flow(&m, X, N, T, za, zb);
    }
    fft_c(X, N, -1);
    return 0;
}

/* ------------------------------------------------------------ adjoints */
/*
 * Reverse mode of the two discrete methods above, for a real loss l of the
 * output field.  A gradient g of a complex quantity x is dl/dRe x + i dl/dIm x,
 * so that dl = Re(conj(g) dx).  For y = c x (c complex): g_x = conj(c) g_y.
 * For y = F[x]: g_x = N F^-1[g_y];  for y = F^-1[x]: g_x = F[g_y] / N.
 * For U = |A|^2 A:  g_A = 2 |A|^2 g_U + A^2 conj(g_U).
 *
 * Parameters are those of the physical segments of the link: segment s of
 * period p is index p n_seg + s (n_periods n_seg of them).  A coefficient
 * enters the method through the integrals of beta2 over [z0, z_j] (the
 * phases of Eq. (6) and of step 7, the linear steps of Eq. (4)) and through
 * sigma(z_j) (Eq. (6)) or int sigma over a step (Eq. (4)).
 */

/* g[P] += w |[za, zb] n segment P| for every physical segment P. */
static void add_overlaps(const fmap* m, double za, double zb, double w, double* g) {
    if (!(zb > za) || w == 0.0) return;
    for (int p = 0; p < m->n_periods; p++) {
        double off = (double)p * m->period;
        for (int s = 0; s < m->n_seg; s++) {
            double a = off, b = off + m->rows[NCOL * s];
            off = b;
            double lo = a > za ? a : za, hi = b < zb ? b : zb;
            if (hi > lo) g[p * m->n_seg + s] += w * (hi - lo);
        }
    }
}

/* Physical segment holding z from the left (side < 0) or the right (side > 0),
 * with the same offset as coef_side; -1 outside the link. */
static int seg_at(const fmap* m, double z, int side) {
    double zz = z + (side > 0 ? 1e-9 : -1e-9) * m->period;
    long p = (long)floor(zz / m->period);
    double u = zz - (double)p * m->period, off = 0.0;
    int s = m->n_seg - 1;
    for (int i = 0; i < m->n_seg; i++) {
        off += m->rows[NCOL * i];
        if (u < off) { s = i; break; }
    }
    if (p < 0 || p >= m->n_periods) return -1;
    return (int)p * m->n_seg + s;
}

/* Reverse mode of one MPA interval: from psi0 = A_hat(z0) and the gradient
 * gX of the interval's output A_hat(z0+L) (after step 7 and the gain),
 * writes the gradient of psi0 to gin and adds the parameter gradients.
 * The forward pass is repeated here with every level kept. */
static int mpa_interval_adjoint(const fmap* m, long N, double T, double z0, double L, int M, int n_tot,
                                const cplx* psi0, const cplx* gX, cplx* gin, double* gsig, double* gb2,
                                int n_threads) {
    const double dz = L / (double)M;
    const size_t nn = (size_t)(M + 1) * (size_t)N;
    const int nthr = n_threads > 0 ? n_threads : ORACLE_MAX_THREADS();
    cplx* psi = (cplx*)malloc(sizeof(cplx) * nn * (size_t)n_tot); /* psi^{(n)}_j */
    cplx* A = (cplx*)malloc(sizeof(cplx) * nn * (size_t)n_tot);   /* A^{(n)}_j(t) */
    cplx* V = (cplx*)malloc(sizeof(cplx) * nn * (size_t)n_tot);   /* V^{(n)}_j */
    cplx* gp = (cplx*)malloc(sizeof(cplx) * nn);                   /* gradient of psi^{(n+1)} */
    cplx* gv = (cplx*)malloc(sizeof(cplx) * nn);                   /* gradient of V^{(n)} */
    cplx* Xo = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    double* I2 = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* I3 = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* sig = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* loss = (double*)malloc(sizeof(double) * (size_t)(M + 1));
    double* s2 = (double*)malloc(sizeof(double) * (size_t)(M + 1));  /* sum_k w^2/2 (.) per node */
    double* hs = (double*)malloc(sizeof(double) * (size_t)(M + 1));  /* d l / d sigma(z_j) */
    int err = 0;
    if (!psi || !A || !V || !gp || !gv || !Xo || !I2 || !I3 || !sig || !loss || !s2 || !hs) err = 3;
    if (!err) {
        for (int j = 0; j <= M; j++) {
            double zj = z0 + dz * (double)j;
            I2[j] = integrate(m, z0, zj, 1);
            I3[j] = integrate(m, z0, zj, 2);
            loss[j] = exp(int_G(m, z0, zj));
            if (j == 0) sig[j] = coef_side(m, zj, 3, +1);
            else if (j == M) sig[j] = coef_side(m, zj, 3, -1);
            else sig[j] = 0.5 * (coef_side(m, zj, 3, -1) + coef_side(m, zj, 3, +1));
            s2[j] = 0.0;
            hs[j] = 0.0;
        }
        /* forward, every level kept */
        for (int j = 0; j <= M; j++) memcpy(psi + (size_t)j * N, psi0, sizeof(cplx) * (size_t)N);
        for (int it = 0; it < n_tot && !err; it++) {
            cplx* P = psi + nn * (size_t)it;
            cplx* Ai = A + nn * (size_t)it;
            cplx* Vi = V + nn * (size_t)it;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr)
            for (int j = 0; j <= M; j++) {
                cplx* a = Ai + (size_t)j * N;
                cplx* v = Vi + (size_t)j * N;
                for (long k = 0; k < N; k++) {
                    double b = beta_of(omega_of(k, N, T), I2[j], I3[j]);
                    a[k] = P[(size_t)j * N + k] * (cos(b) + I * sin(b)) * loss[j];
                }
                fft_c(a, N, -1);
                for (long n = 0; n < N; n++) {
                    double q = creal(a[n]) * creal(a[n]) + cimag(a[n]) * cimag(a[n]);
                    v[n] = a[n] * q;
                }
                fft_c(v, N, +1);
                for (long k = 0; k < N; k++) {
                    double b = beta_of(omega_of(k, N, T), I2[j], I3[j]);
                    v[k] = sig[j] * dz * v[k] * (cos(b) - I * sin(b)) / loss[j];
                }
            }
            if (it + 1 < n_tot) {
                cplx* Pn = psi + nn * (size_t)(it + 1);
                memcpy(Pn, psi0, sizeof(cplx) * (size_t)N);
                for (long k = 0; k < N; k++) {
                    cplx run = 0.5 * Vi[k];
                    for (int l = 1; l <= M; l++) {
                        cplx vl = Vi[(size_t)l * N + k];
                        Pn[(size_t)l * N + k] = psi0[k] + I * (run + 0.5 * vl);
                        run += vl;
                    }
                }
            }
        }
    }
    if (!err) {
        /* output of the interval: step 7 on psi^{(n_tot)}_M, then the gain */
        const cplx* Vl = V + nn * (size_t)(n_tot - 1);
        double I2L = integrate(m, z0, z0 + L, 1), I3L = integrate(m, z0, z0 + L, 2);
        double g = exp(int_G(m, z0, z0 + L) + (double)n_amps(m, z0, z0 + L) * m->z_a * m->gamma);
        double srec = 0.0;
        memset(gp, 0, sizeof(cplx) * nn);
        for (long k = 0; k < N; k++) {
            cplx run = 0.5 * Vl[k];
            for (int l = 1; l < M; l++) run += Vl[(size_t)l * N + k];
            cplx psiM = psi0[k] + I * (run + 0.5 * Vl[(size_t)M * N + k]);
            double w = omega_of(k, N, T), b = beta_of(w, I2L, I3L);
            cplx e = (cos(b) + I * sin(b)) * g;
            Xo[k] = psiM * e;
            gp[(size_t)M * N + k] = conj(e) * gX[k];
            /* d Xo / d beta = i Xo d beta */
            srec += 0.5 * w * w * creal(conj(gX[k]) * I * Xo[k]);
        }
        add_overlaps(m, z0, z0 + L, srec, gb2);
        memset(gin, 0, sizeof(cplx) * (size_t)N);
        for (int it = n_tot - 1; it >= 0; it--) {
            const cplx* P = psi + nn * (size_t)it;
            const cplx* Ai = A + nn * (size_t)it;
            const cplx* Vi = V + nn * (size_t)it;
            /* step 5 reversed: psi_l = psi_0 + i (V_0/2 + sum_{0<j<l} V_j + V_l/2),
             * every psi_l also carries psi_0 itself */
            for (long k = 0; k < N; k++) {
                cplx tail = 0.0; /* sum_{l>j} g_psi_l */
                for (int j = M; j >= 0; j--) {
                    cplx gl = gp[(size_t)j * N + k];
                    gin[k] += gl;
                    cplx c = (j == 0) ? 0.5 * tail : tail + 0.5 * gl;
                    gv[(size_t)j * N + k] = -I * c;
                    if (j > 0) tail += gl;
                }
            }
            /* steps 4..2 reversed at every node */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr)
            for (int j = 0; j <= M; j++) {
                cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)N);
                if (!w) { err = 3; continue; }
                const cplx* a = Ai + (size_t)j * N;
                const cplx* gvj = gv + (size_t)j * N;
                const cplx* vj = Vi + (size_t)j * N;
                double bpost = 0.0, bpre = 0.0, hsig = 0.0;
                /* V_j = sig_j dz F[U] e^{-i beta} / loss_j */
                for (long k = 0; k < N; k++) {
                    double om = omega_of(k, N, T), b = beta_of(om, I2[j], I3[j]);
                    bpost += 0.5 * om * om * creal(conj(gvj[k]) * (-I) * vj[k]);
                    w[k] = dz * (cos(b) + I * sin(b)) / loss[j] * gvj[k]; /* gradient of F[U] / sig_j */
                }
                fft_c(w, N, -1);
                for (long n = 0; n < N; n++) {
                    cplx gu = w[n] * (double)N; /* gradient of U over sig_j */
                    cplx an = a[n];
                    double q = creal(an) * creal(an) + cimag(an) * cimag(an);
                    hsig += creal(conj(gu) * (an * q));
                    w[n] = sig[j] * (2.0 * q * gu + an * an * conj(gu)); /* gradient of A */
                }
                fft_c(w, N, +1);
                for (long k = 0; k < N; k++) {
                    double om = omega_of(k, N, T), b = beta_of(om, I2[j], I3[j]);
                    cplx gP = w[k] / (double)N; /* gradient of psi_j e^{i beta} loss_j */
                    cplx e = (cos(b) + I * sin(b)) * loss[j];
                    cplx Pk = P[(size_t)j * N + k] * e;
                    bpre += 0.5 * om * om * creal(conj(gP) * I * Pk);
                    w[k] = conj(e) * gP;
                }
                memcpy(gp + (size_t)j * N, w, sizeof(cplx) * (size_t)N); /* gradient of psi^{(it)}_j */
                s2[j] += bpost + bpre;
                hs[j] += hsig;
                free(w);
            }
            if (err) break;
        }
        if (!err) {
            /* psi^{(0)}_j = psi_0 at every node */
            for (int j = 0; j <= M; j++)
                for (long k = 0; k < N; k++) gin[k] += gp[(size_t)j * N + k];
            /* parameters: beta2 through int_{z0}^{z_j} beta2, sigma through sigma(z_j) */
            for (int j = 0; j <= M; j++) {
                double zj = z0 + dz * (double)j;
                add_overlaps(m, z0, zj, s2[j], gb2);
                int sl = seg_at(m, zj, -1), sr = seg_at(m, zj, +1);
                if (j == 0) { if (sr >= 0) gsig[sr] += hs[j]; }
                else if (j == M) { if (sl >= 0) gsig[sl] += hs[j]; }
                else {
                    if (sl >= 0) gsig[sl] += 0.5 * hs[j];
                    if (sr >= 0) gsig[sr] += 0.5 * hs[j];
                }
            }
        }
    }
    free(psi); free(A); free(V); free(gp); free(gv); free(Xo);
    free(I2); free(I3); free(sig); free(loss); free(s2); free(hs);
    return err;
}

static int mpa_grid(const fmap* m, double z_from, double z_to, double L, long* n_int) {
    if (check_span(m, z_from, z_to)) return 2;
    double cnt = (z_to - z_from) / L;
    long n = lround(cnt);
    if (fabs(cnt - (double)n) > 1e-9 * (cnt > 1.0 ? cnt : 1.0)) return 2;
    for (long q = 0; q < n; q++) {
        double a = z_from + L * (double)q, b = z_from + L * (double)(q + 1);
        if (amp_inside(m, a, b)) return 2;
    }
    *n_int = n;
    return 0;
}

int oracle_mpa_adjoint(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
                       long N, double T, double z_from, double z_to, double L, int M, int n_tot,
                       const double* field_in, const double* grad_out, double* grad_in,
                       double* grad_sigma, double* grad_beta2, double* field_out, int n_threads) {
    if (!is_pow2(N)) return 1;
    if (M < 1 || n_tot < 1 || !(L > 0.0) || !(T > 0.0) || n_seg < 1 || n_periods < 1) return 4;
    fmap m = make_map(seg_rows, n_seg, gamma, z_a, n_periods);
    long n_int = 0;
    int err = mpa_grid(&m, z_from, z_to, L, &n_int);
    if (err) return err;
    const int n_phys = n_periods * n_seg;
    for (int s = 0; s < n_phys; s++) grad_sigma[s] = grad_beta2[s] = 0.0;
    cplx* ck = (cplx*)malloc(sizeof(cplx) * (size_t)N * (size_t)(n_int + 1)); /* A_hat at interval starts */
    cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* gn = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    if (!ck || !g || !gn) { free(ck); free(g); free(gn); return 3; }
    /* forward with a checkpoint per interval */
    memcpy(ck, field_in, sizeof(cplx) * (size_t)N);
    fft_c(ck, N, +1);
    for (long q = 0; q < n_int && !err; q++) {
        double z0 = z_from + L * (double)q;
        cplx* X = ck + (size_t)N * (size_t)q;
        cplx* Y = ck + (size_t)N * (size_t)(q + 1);
        err = mpa_interval(&m, N, T, z0, L, M, n_tot, X, Y, n_threads);
        if (err) break;
        double I2 = integrate(&m, z0, z0 + L, 1), I3 = integrate(&m, z0, z0 + L, 2);
        double gg = exp(int_G(&m, z0, z0 + L) + (double)n_amps(&m, z0, z0 + L) * m.z_a * m.gamma);
        for (long k = 0; k < N; k++) {
            double b = beta_of(omega_of(k, N, T), I2, I3);
            Y[k] *= (cos(b) + I * sin(b)) * gg;
        }
    }
    if (!err && field_out) {
        memcpy(field_out, ck + (size_t)N * (size_t)n_int, sizeof(cplx) * (size_t)N);
        fft_c((cplx*)field_out, N, -1);
    }
    /* output A = F^-1[A_hat]  =>  g_{A_hat} = F[g_A] / N */
    memcpy(g, grad_out, sizeof(cplx) * (size_t)N);
    fft_c(g, N, +1);
    for (long k = 0; k < N; k++) g[k] /= (double)N;
    for (long q = n_int - 1; q >= 0 && !err; q--) {
        double z0 = z_from + L * (double)q;
        err = mpa_interval_adjoint(&m, N, T, z0, L, M, n_tot, ck + (size_t)N * (size_t)q, g, gn, grad_sigma,
                                   grad_beta2, n_threads);
        memcpy(g, gn, sizeof(cplx) * (size_t)N);
    }
    /* input A_hat = F[A]  =>  g_A = N F^-1[g_{A_hat}] */
    if (!err) {
        fft_c(g, N, -1);
        for (long k = 0; k < N; k++) ((cplx*)grad_in)[k] = g[k] * (double)N;
    }
    free(ck); free(g); free(gn);
    return err;
}

/* Reverse mode of the split-step of Eq. (4), same conventions. */
int oracle_ss_adjoint(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
                      long N, double T, double z_from, double z_to, double dz,
                      const double* field_in, const double* grad_out, double* grad_in,
                      double* grad_sigma, double* grad_beta2, double* field_out) {
    if (!is_pow2(N)) return 1;
    if (!(dz > 0.0) || !(T > 0.0) || n_seg < 1 || n_periods < 1) return 4;
    fmap m = make_map(seg_rows, n_seg, gamma, z_a, n_periods);
    if (check_span(&m, z_from, z_to)) return 2;
    double cnt = (z_to - z_from) / dz;
    long K = lround(cnt);
    if (K < 1 || fabs(cnt - (double)K) > 1e-9 * (cnt > 1.0 ? cnt : 1.0)) return 2;
    const int n_phys = n_periods * n_seg;
    for (int s = 0; s < n_phys; s++) grad_sigma[s] = grad_beta2[s] = 0.0;
    /* trajectory: the time-domain field entering each nonlinear step */
    cplx* traj = (cplx*)malloc(sizeof(cplx) * (size_t)N * (size_t)K);
    cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    double* ls = (double*)malloc(sizeof(double) * (size_t)(K + 1) * 2); /* linear step ends */
    double* sk = (double*)malloc(sizeof(double) * (size_t)K);
    if (!traj || !X || !ls || !sk) { free(traj); free(X); free(ls); free(sk); return 3; }
    double za = z_from, zb = z_from + 0.5 * dz;
    ls[0] = za; ls[1] = zb;
    for (long k = 0; k < K; k++) {
        double zk = z_from + dz * (double)k;
        sk[k] = integrate(&m, zk, zk + dz, 3);
        za = zb;
        zb = (k == K - 1) ? z_to : zb + dz;
        ls[2 * (k + 1)] = za;
        ls[2 * (k + 1) + 1] = zb;
    }
    memcpy(X, field_in, sizeof(cplx) * (size_t)N);
    fft_c(X, N, +1);
    linear_flow(&m, X, N, T, ls[0], ls[1]);
    for (long k = 0; k < K; k++) {
        fft_c(X, N, -1);
        memcpy(traj + (size_t)N * (size_t)k, X, sizeof(cplx) * (size_t)N);
        for (long n = 0; n < N; n++) {
            double p = creal(X[n]) * creal(X[n]) + cimag(X[n]) * cimag(X[n]);
            X[n] *= cos(sk[k] * p) + I * sin(sk[k] * p);
        }
        fft_c(X, N, +1);
        linear_flow(&m, X, N, T, ls[2 * (k + 1)], ls[2 * (k + 1) + 1]);
    }
    if (field_out) {
        memcpy(field_out, X, sizeof(cplx) * (size_t)N);
        fft_c((cplx*)field_out, N, -1);
    }
    /* reverse: g is the gradient of the spectrum after linear step k+1 */
    cplx* g = X;
    memcpy(g, grad_out, sizeof(cplx) * (size_t)N);
    fft_c(g, N, +1);
    for (long n = 0; n < N; n++) g[n] /= (double)N;
    for (long k = K; k >= 0; k--) {
        /* linear step over [ls[2k], ls[2k+1]]: y = H x */
        double a = ls[2 * k], b = ls[2 * k + 1];
        double I2 = integrate(&m, a, b, 1), I3 = integrate(&m, a, b, 2);
        double gg = exp(int_G(&m, a, b) + (double)n_amps(&m, a, b) * m.z_a * m.gamma);
        /* y = H x with x the spectrum before the step: recompute it */
        cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)N);
        if (!x) { free(traj); free(X); free(ls); free(sk); return 3; }
        if (k == 0) {
            memcpy(x, field_in, sizeof(cplx) * (size_t)N);
            fft_c(x, N, +1);
        } else {
            const cplx* t = traj + (size_t)N * (size_t)(k - 1);
            for (long n = 0; n < N; n++) {
                double p = creal(t[n]) * creal(t[n]) + cimag(t[n]) * cimag(t[n]);
                x[n] = t[n] * (cos(sk[k - 1] * p) + I * sin(sk[k - 1] * p));
            }
            fft_c(x, N, +1);
        }
        double sb = 0.0;
        for (long n = 0; n < N; n++) {
            double om = omega_of(n, N, T), be = beta_of(om, I2, I3);
            cplx h = (cos(be) + I * sin(be)) * gg;
            sb += 0.5 * om * om * creal(conj(g[n]) * I * h * x[n]);
            g[n] = conj(h) * g[n];
        }
        add_overlaps(&m, a, b, sb, grad_beta2);
        free(x);
        if (k == 0) break;
        /* nonlinear step k-1 on the time-domain field t: y = t e^{i s |t|^2} */
        const cplx* t = traj + (size_t)N * (size_t)(k - 1);
        fft_c(g, N, -1);
        for (long n = 0; n < N; n++) g[n] *= (double)N; /* gradient of the time-domain y */
        double gs = 0.0;
        for (long n = 0; n < N; n++) {
            double p = creal(t[n]) * creal(t[n]) + cimag(t[n]) * cimag(t[n]);
            cplx e = cos(sk[k - 1] * p) + I * sin(sk[k - 1] * p);
            cplx y = t[n] * e;
            double c = creal(conj(g[n]) * I * y); /* d l / d phase */
            gs += c * p;
            g[n] = conj(e) * g[n] + 2.0 * c * sk[k - 1] * t[n];
        }
        double zk = z_from + dz * (double)(k - 1);
        add_overlaps(&m, zk, zk + dz, gs, grad_sigma);
        fft_c(g, N, +1);
        for (long n = 0; n < N; n++) g[n] /= (double)N; /* gradient of the spectrum before F^-1 */
    }
    fft_c(g, N, -1);
    for (long n = 0; n < N; n++) ((cplx*)grad_in)[n] = g[n] * (double)N;
    free(traj); free(X); free(ls); free(sk);
    return 0;
}
