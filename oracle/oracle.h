/*
 * FP64 CPU oracle for the massively parallel algorithm (MPA) and the
 * split-step (SS) method for the dispersion-managed NLSE, Eq. (1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA library: the fiber map is
 * re-interpreted here from the same plain segment rows, the Fourier transform
 * is this file's own radix-2 FFT, and every phase is evaluated directly in
 * FP64 from its definition.
 *
 * Conventions (Eq. (1) and the Fourier transform that follows it):
 *   forward  F[x]_k     = sum_n x_n exp(+2 pi i k n / N)      (unnormalised)
 *   inverse  F^-1[X]_n  = (1/N) sum_k X_k exp(-2 pi i k n / N)
 *   omega_k  = 2 pi k' / T, k' = k for k < N/2, k - N otherwise
 *   beta(omega, za, zb) = omega^2/2 int_za^zb beta2 + omega^3/6 int_za^zb beta3
 *   G = -gamma + g between amplifiers (g: the distributed gain of the
 *   segment); amplifier k (z_k = k z_a, k >= 1) multiplies
 *   the field by exp(z_a gamma) when the propagation crosses z_k, i.e. for
 *   z_k in (z_from, z_to].
 *
 * Fields are interleaved complex128 (re, im) arrays of length 2N.
 * Segment rows are n_seg x 5 doubles: length_km, beta2, beta3, sigma,
 * gain (distributed amplitude gain, 1/km).
 *
 * Return codes: 0 ok; 1 N not a power of two >= 2; 2 z-grid inconsistent
 * (interval count not whole, amplifier strictly inside an MPA interval, or
 * beyond the end of the link); 3 out of memory; 4 bad argument.
 */
#ifndef MPA_ORACLE_H
#define MPA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* In-place FFT of N interleaved complex128 values.  sign=+1: F, sign=-1: F^-1. */
int oracle_fft(double* x, long N, int sign);

/* MPA, Eq. (6) with steps 1-7: propagate the time-domain field in place from
 * z_from to z_to in intervals of length L, each with M+1 nodes and n_tot
 * Picard iterations.  n_threads <= 0 lets OpenMP choose; the number of
 * threads actually used is written to *threads_used (may be NULL). */
int oracle_mpa(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
               long N, double T, double z_from, double z_to, double L, int M, int n_tot,
               double* field, int n_threads, int* threads_used);

/* Symmetric split-step, Eq. (4): half linear step, then M x (nonlinear phase
 * rotation, linear step) with the last linear step halved. */
int oracle_ss(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
              long N, double T, double z_from, double z_to, double dz, double* field);

/* The MPA outputs of one interval [z0, z0+L] from a given spectrum psi0
 * (N complex, natural frequency order): the node-n_tot spectrum psi_M
 * before the reconstruction of step 7.  Exposed for the parity tests of
 * single intervals. */
int oracle_mpa_interval(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
                        long N, double T, double z0, double L, int M, int n_tot,
                        const double* psi0, double* psiM, int n_threads);

/* Reverse mode of oracle_mpa for a real loss l of the output field.  Given
 * the input field and g_out = dl/dRe A_out + i dl/dIm A_out, writes the
 * gradient of the input field (same convention), and dl/dsigma and
 * dl/dbeta2 of every physical segment (n_periods x n_seg values, segment s
 * of period p at p n_seg + s), and the output field if field_out != NULL.
 * Forward with a checkpoint per interval; each interval's levels are
 * recomputed and walked backwards (MPA steps 7..2, Eq. (6)). */
int oracle_mpa_adjoint(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
                       long N, double T, double z_from, double z_to, double L, int M, int n_tot,
                       const double* field_in, const double* grad_out, double* grad_in,
                       double* grad_sigma, double* grad_beta2, double* field_out, int n_threads);

/* Reverse mode of oracle_ss (Eq. (4)), same arguments and conventions. */
int oracle_ss_adjoint(const double* seg_rows, int n_seg, double gamma, double z_a, int n_periods,
                      long N, double T, double z_from, double z_to, double dz,
                      const double* field_in, const double* grad_out, double* grad_in,
                      double* grad_sigma, double* grad_beta2, double* field_out);

#ifdef __cplusplus
}
#endif
#endif
