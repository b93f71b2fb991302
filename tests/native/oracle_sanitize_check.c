/*
 * Host-side memory and undefined-behaviour check of the FP64 oracle: this
 * driver links oracle.c and is compiled with AddressSanitizer and
 * UndefinedBehaviorSanitizer (-fsanitize=address,undefined,
 * -fno-sanitize-recover=all), so any out-of-bounds access, use after free,
 * leak, signed overflow or misaligned access in the oracle ends the run with
 * a report and a non-zero exit.  It calls every exported entry point on
 * small cases (N = 2 .. 256; single and multi-segment maps, amplifiers at
 * interval ends, one and two threads, field_out NULL or not) and on each of
 * its argument errors, and checks the return codes and that every output is
 * finite.  The values themselves are pinned by the Python oracle tests.
 *
 * Build (done by tests/test_oracle_sanitize.py):
 *   gcc -std=c11 -O1 -g -fopenmp -fsanitize=address,undefined
 *       -fno-sanitize-recover=all -fno-omit-frame-pointer -I oracle
 *       tests/native/oracle_sanitize_check.c oracle/oracle.c -lm
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static int failures = 0;

#define EXPECT(cond, ...)                            \
    do {                                             \
        if (!(cond)) {                               \
            fprintf(stderr, "FAIL %s:%d: ", __FILE__, __LINE__); \
            fprintf(stderr, __VA_ARGS__);            \
            fputc('\n', stderr);                     \
            failures++;                              \
        }                                            \
    } while (0)

static int all_finite(const double* x, long n) {
    for (long i = 0; i < n; i++)
        if (!isfinite(x[i])) return 0;
    return 1;
}

/* interleaved complex field: a chirped Gaussian plus a displaced one */
static double* make_field(long N, double T) {
    double* a = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    for (long n = 0; n < N; n++) {
        double t = ((double)n - 0.5 * (double)N) * T / (double)N;
        double env = 0.6 * exp(-0.5 * t * t), env2 = 0.4 * exp(-0.5 * (t - 3.0) * (t - 3.0));
        a[2 * n] = env * cos(0.3 * t) + env2;
        a[2 * n + 1] = env * sin(0.3 * t);
    }
    return a;
}

/* two segments per period: {length, beta2, beta3, sigma, gain} */
static const double ROWS2[10] = {0.6, -1.0, 0.1, 1.0, 0.0, 0.4, 2.0, 0.05, 0.7, 0.02};
static const double ROWS1[5] = {1.0, -1.0, 0.0, 1.0, 0.0};

static void check_fft(void) {
    double x[2 * 6] = {0};
    EXPECT(oracle_fft(x, 6, +1) == 1, "fft of a non-power-of-two length must return 1");
    EXPECT(oracle_fft(x, 0, +1) == 1, "fft of length 0 must return 1");
    for (long N = 2; N <= 256; N *= 2) {
        double* a = make_field(N, 16.0);
        double* b = (double*)malloc(sizeof(double) * 2 * (size_t)N);
        memcpy(b, a, sizeof(double) * 2 * (size_t)N);
        EXPECT(oracle_fft(a, N, +1) == 0, "fft N=%ld", N);
        EXPECT(oracle_fft(a, N, -1) == 0, "inverse fft N=%ld", N);
        double err = 0.0;
        for (long i = 0; i < 2 * N; i++) err = fmax(err, fabs(a[i] - b[i]));
        EXPECT(err < 1e-12, "fft round trip N=%ld: %g", N, err);
        free(a);
        free(b);
    }
}

static void check_mpa(void) {
    const double T = 16.0, gamma = 0.05, z_a = 1.0;
    for (long N = 2; N <= 256; N *= 4) {
        for (int n_tot = 1; n_tot <= 3; n_tot++) {
            for (int threads = 1; threads <= 2; threads++) {
                double* a = make_field(N, T);
                int used = -1;
                /* 2 km over a 1-km period with amplifiers at 1 km and 2 km */
                int rc = oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.0, 2.0, 0.5, 3, n_tot, a, threads, &used);
                EXPECT(rc == 0 && used == threads, "mpa N=%ld n=%d threads=%d: rc %d used %d", N, n_tot, threads, rc,
                       used);
                EXPECT(all_finite(a, 2 * N), "mpa output finite N=%ld", N);
                free(a);
            }
        }
    }
    long N = 64;
    double* a = make_field(N, T);
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.5, 0.5, 0.5, 2, 2, a, 1, NULL) == 0, "empty range");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.0, 1.0, 1.0, 1, 1, a, 1, NULL) == 0, "M = 1");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, 48, T, 0.0, 1.0, 0.5, 2, 2, a, 1, NULL) == 1, "N not 2^k");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.0, 1.0, 0.3, 2, 2, a, 1, NULL) == 2, "interval count");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.5, 1.5, 1.0, 2, 2, a, 1, NULL) == 2, "amplifier inside");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.0, 3.0, 0.5, 2, 2, a, 1, NULL) == 2, "beyond the link");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.0, 1.0, 0.5, 0, 2, a, 1, NULL) == 4, "M = 0");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, T, 0.0, 1.0, 0.5, 2, 0, a, 1, NULL) == 4, "n_tot = 0");
    EXPECT(oracle_mpa(ROWS2, 2, gamma, z_a, 2, N, -1.0, 0.0, 1.0, 0.5, 2, 2, a, 1, NULL) == 4, "T < 0");
    EXPECT(oracle_mpa(ROWS2, 0, gamma, z_a, 2, N, T, 0.0, 1.0, 0.5, 2, 2, a, 1, NULL) == 4, "no segments");
    EXPECT(all_finite(a, 2 * N), "field after the rejected calls");
    free(a);
}

static void check_mpa_interval(void) {
    const double T = 16.0;
    for (long N = 2; N <= 256; N *= 4) {
        double* p0 = make_field(N, T);
        double* pm = (double*)malloc(sizeof(double) * 2 * (size_t)N);
        oracle_fft(p0, N, +1);
        /* an interval that starts mid-period and crosses a segment boundary */
        EXPECT(oracle_mpa_interval(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.25, 0.5, 4, 3, p0, pm, 2) == 0,
               "mpa_interval N=%ld", N);
        EXPECT(all_finite(pm, 2 * N), "mpa_interval output finite N=%ld", N);
        EXPECT(oracle_mpa_interval(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.25, 0.0, 4, 3, p0, pm, 1) == 4, "L = 0");
        free(p0);
        free(pm);
    }
}

static void check_ss(void) {
    const double T = 16.0;
    for (long N = 2; N <= 256; N *= 4) {
        double* a = make_field(N, T);
        EXPECT(oracle_ss(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.0, 2.0, 0.05, a) == 0, "ss N=%ld", N);
        EXPECT(all_finite(a, 2 * N), "ss output finite N=%ld", N);
        EXPECT(oracle_ss(ROWS1, 1, 0.0, 1.0, 1, N, T, 0.0, 1.0, 0.25, a) == 0, "ss single segment N=%ld", N);
        free(a);
    }
    double* a = make_field(64, T);
    EXPECT(oracle_ss(ROWS2, 2, 0.05, 1.0, 2, 64, T, 0.0, 1.0, 0.3, a) == 2, "ss step count");
    EXPECT(oracle_ss(ROWS2, 2, 0.05, 1.0, 2, 64, T, 0.0, 0.0, 0.1, a) == 2, "ss zero steps");
    EXPECT(oracle_ss(ROWS2, 2, 0.05, 1.0, 2, 64, T, 0.0, 1.0, 0.0, a) == 4, "ss dz = 0");
    EXPECT(oracle_ss(ROWS2, 2, 0.05, 1.0, 2, 100, T, 0.0, 1.0, 0.1, a) == 1, "ss N not 2^k");
    free(a);
}

static void check_adjoints(void) {
    const double T = 16.0;
    const int n_phys = 2 * 2;
    for (long N = 2; N <= 256; N *= 4) {
        double* a = make_field(N, T);
        double* g = make_field(N, T);
        double* gi = (double*)malloc(sizeof(double) * 2 * (size_t)N);
        double* out = (double*)malloc(sizeof(double) * 2 * (size_t)N);
        double gs[4], gb[4];
        for (int with_out = 0; with_out <= 1; with_out++) {
            int rc = oracle_mpa_adjoint(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.0, 2.0, 0.5, 3, 2, a, g, gi, gs, gb,
                                        with_out ? out : NULL, 2);
            EXPECT(rc == 0, "mpa_adjoint N=%ld out=%d: rc %d", N, with_out, rc);
            EXPECT(all_finite(gi, 2 * N) && all_finite(gs, n_phys) && all_finite(gb, n_phys), "mpa_adjoint finite");
            rc = oracle_ss_adjoint(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.0, 2.0, 0.1, a, g, gi, gs, gb,
                                   with_out ? out : NULL);
            EXPECT(rc == 0, "ss_adjoint N=%ld out=%d: rc %d", N, with_out, rc);
            EXPECT(all_finite(gi, 2 * N) && all_finite(gs, n_phys) && all_finite(gb, n_phys), "ss_adjoint finite");
            if (with_out) EXPECT(all_finite(out, 2 * N), "adjoint forward output finite");
        }
        /* a range that starts and ends inside the link, not at z = 0 */
        EXPECT(oracle_mpa_adjoint(ROWS2, 2, 0.05, 1.0, 2, N, T, 1.0, 2.0, 0.5, 2, 1, a, g, gi, gs, gb, out, 1) == 0,
               "mpa_adjoint from 1 km");
        free(a);
        free(g);
        free(gi);
        free(out);
    }
    long N = 64;
    double* a = make_field(N, T);
    double* g = make_field(N, T);
    double* gi = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double gs[4], gb[4];
    EXPECT(oracle_mpa_adjoint(ROWS2, 2, 0.05, 1.0, 0, N, T, 0.0, 1.0, 0.5, 2, 2, a, g, gi, gs, gb, NULL, 1) == 4,
           "mpa_adjoint without periods");
    EXPECT(oracle_mpa_adjoint(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.5, 1.5, 1.0, 2, 2, a, g, gi, gs, gb, NULL, 1) == 2,
           "mpa_adjoint amplifier inside");
    EXPECT(oracle_ss_adjoint(ROWS2, 2, 0.05, 1.0, 2, N, T, 0.0, 1.0, 0.3, a, g, gi, gs, gb, NULL) == 2,
           "ss_adjoint step count");
    EXPECT(oracle_ss_adjoint(ROWS2, 2, 0.05, 1.0, 2, 12, T, 0.0, 1.0, 0.1, a, g, gi, gs, gb, NULL) == 1,
           "ss_adjoint N not 2^k");
    free(a);
    free(g);
    free(gi);
}

int main(void) {
    check_fft();
    check_mpa();
    check_mpa_interval();
    check_ss();
    check_adjoints();
    if (failures) {
        fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    printf("oracle sanitizer checks passed\n");
    return 0;
}
