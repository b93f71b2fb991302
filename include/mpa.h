/*
 * mpa.h -- C ABI of the GB300 (sm_103a) implementation of the massively
 * parallel algorithm (MPA) for the dispersion-managed WDM nonlinear
 * Schroedinger equation (Korotkevich & Lushnikov, arXiv:1101.0086), with the
 * symmetric split-step (SS) method of Eq. (4) on the same GPU.
 *
 * Physics (Eq. (1)):
 *   i A_z - beta2(z)/2 A_tt - i beta3(z)/6 A_ttt + sigma(z)|A|^2 A = i G(z) A,
 *   G(z) = -gamma + (exp(z_a gamma) - 1) sum_k delta(z - k z_a).
 * Units: t in ps, z in km, beta2 in ps^2/km, beta3 in ps^3/km,
 * sigma in 1/(W km), |A|^2 in W, gamma (amplitude loss) in 1/km.
 *
 * Fourier convention (text after Eq. (1)): A_hat(w) = int A(t) exp(+i w t) dt,
 * discretised as F[x]_k = sum_n x_n exp(+2 pi i k n/N) with
 * w_k = 2 pi k'/T, k' = k (k < N/2) or k - N (k >= N/2).
 *
 * Field layout: A(t_n), t_n = n T/N, n = 0..N-1, interleaved (re, im):
 * complex64 (float2) for MPA_FP32, complex128 (double2) for MPA_FP64.
 * All field and workspace pointers are DEVICE pointers owned by the caller;
 * the library allocates no device memory: scratch and tables live in the
 * caller's workspace.
 * Streams are cudaStream_t values passed as void* (NULL = legacy default
 * stream).  Calls are stream-ordered and asynchronous unless stated.
 *
 * Errors: every entry point returns an int status (MPA_OK = 0).  Argument
 * and grid checks are synchronous; a CUDA launch or copy failure returns
 * MPA_ERR_CUDA; a host allocation that fails (plan and batch tables, the
 * per-interval schedules of a propagation or gradient) returns
 * MPA_ERR_HOST_MEMORY and leaves no partly built object behind.  Nothing
 * aborts or throws across the ABI.
 */
#ifndef MPA_H
#define MPA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MPA_API __attribute__((visibility("default")))
#else
#define MPA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MPA_OK = 0,
    MPA_ERR_INVALID_ARG = 1,   /* NULL pointer, non-positive size, bad enum */
    MPA_ERR_UNSUPPORTED_N = 2, /* N not a power of two in [2^8, 2^25] (2^24 for FP64) */
    MPA_ERR_WORKSPACE = 3,     /* workspace missing or smaller than required */
    MPA_ERR_CUDA = 4,          /* a CUDA call failed (see mpa_last_cuda_error) */
    MPA_ERR_GRID = 5,          /* z-grid inconsistent with the fiber map (see each call) */
    MPA_ERR_NONFINITE = 6,     /* a NaN/Inf was produced (mpa_plan_status, mpa_batch_status) */
    MPA_ERR_DIVERGED = 7,      /* the Picard iteration did not contract (mpa_plan_status, mpa_batch_status) */
    MPA_ERR_SCALES = 8,        /* scales outside the weakly nonlinear regime (mpa_plan_check_scales) */
    MPA_ERR_TIMEOUT = 9,       /* a bounded wait of a persistent kernel ran out (mpa_plan_status, mpa_batch_status) */
    MPA_ERR_BOUNDS = 10,       /* debug build: an access outside the checked range was skipped (mpa_plan_status) */
    MPA_ERR_HOST_MEMORY = 11   /* a host allocation failed (or a table too large for the host was asked for) */
};

enum { MPA_FP32 = 0, MPA_FP64 = 1 };

/* Launch schedule of the MPA steps within an interval.  LEVEL: the paper's
 * order, every node of an iteration, then the next iteration (memory
 * (M+1) N samples).  WAVEFRONT: node blocks advance through the iterations
 * one step at a time, the forward and inverse column transforms of
 * consecutive iterations and the trapezoid sums fused in one kernel (FP32,
 * memory about 3 n_iter N samples + 256 MiB).  Both compute Eq. (6); they
 * differ only in FP32 summation order.  WAVEFRONT needs FP32, N >= 2^14 and
 * n_iter <= 8.  AUTO picks LEVEL, the faster of the two on GB300 at the
 * benchmark sizes (the wavefront saves memory, not time). */
enum { MPA_SCHEDULE_AUTO = 0, MPA_SCHEDULE_LEVEL = 1, MPA_SCHEDULE_WAVEFRONT = 2 };

typedef void* mpa_stream; /* cudaStream_t */

/* One piece of the dispersion-management period with constant coefficients.
 * gain_per_km is a distributed amplitude gain g of the piece (e.g. a
 * Raman-pumped span; the paper notes that distributed amplification can be
 * included in G): between lumped amplifiers G(z) = g(z) - gamma. */
typedef struct {
    double length_km;
    double beta2_ps2_per_km;
    double beta3_ps3_per_km;
    double sigma_per_W_km;
    double gain_per_km;
} mpa_segment;

/* Periodic fiber map (Eq. (1): beta2, beta3 periodic in z; sigma and the
 * distributed gain per segment).
 * segments[0..n_segments) form one period, repeated n_periods times.
 * Lumped amplifiers at z_k = k z_a_km, k >= 1, multiply the field by
 * exp(z_a gamma) when the propagation crosses z_k (z_k in (z_from, z_to]).
 * z_a_km <= 0 disables amplifiers.  The map is copied by the calls that take
 * it; the caller keeps ownership of `segments`. */
typedef struct {
    const mpa_segment* segments;
    int32_t n_segments;
    double gamma_per_km;
    double z_a_km;
    int32_t n_periods;
} mpa_fiber_map;

/* gamma_per_km of a fiber whose POWER loss is db_per_km dB/km: G = -gamma in
 * Eq. (1) acts on the amplitude, so |A|^2 decays as exp(-2 gamma z) =
 * 10^(-db_per_km z / 10), i.e. gamma = db_per_km ln(10) / 20.  Host only;
 * never fails (NaN in, NaN out). */
MPA_API double mpa_gamma_from_db_per_km(double db_per_km);

/* MPA discretisation (MPA steps 1-7 and Eq. (6)): intervals of length L_km,
 * each with M+1 equally spaced nodes and n_iter Picard iterations. */
typedef struct {
    int64_t N;         /* Fourier modes, power of two */
    double T_ps;       /* time window */
    double L_km;       /* interval length; must divide the DM period (at most 2^20 intervals per period,
                          else MPA_ERR_GRID) or be a multiple of it */
    int32_t M;         /* intervals of the z-quadrature per interval (M+1 nodes), 1 <= M <= 2^24 */
    int32_t n_iter;    /* n_tot, Picard iterations per interval (>= 1) */
    int32_t precision; /* MPA_FP32 (FFT/nonlinearity in FP32, phase exact, Kahan sums, FP64 state) or MPA_FP64 */
    int32_t schedule;  /* MPA_SCHEDULE_* (0 = AUTO); WAVEFRONT where unsupported is MPA_ERR_INVALID_ARG */
} mpa_plan_params;

typedef struct mpa_plan mpa_plan;

/* Create a plan (host only, no CUDA call).  Validates N, T, L, M, n_iter
 * and the map; precomputes on the host, for every distinct interval start
 * within the DM period, the per-node constants of Eq. (6): the exact
 * fixed-point phase coefficients of beta(w, z_j), the loss factor
 * exp(int G) and the trapezoid weight sigma(z_j) dz.  *out receives the plan. */
MPA_API int mpa_plan_create(const mpa_fiber_map* map, const mpa_plan_params* params, mpa_plan** out);

/* Bytes of device workspace the plan needs (caller allocates, >= 256-B aligned). */
MPA_API int mpa_plan_workspace_size(const mpa_plan* plan, size_t* bytes);

/* Attach caller-owned device workspace and upload the node tables
 * (synchronous).  The workspace must stay valid while the plan is used. */
MPA_API int mpa_plan_set_workspace(mpa_plan* plan, void* workspace, size_t bytes);

/* MPA propagation (MPA steps 1-7 per interval, interval marching of the text
 * before step 1): the time-domain field is propagated in place from
 * z_from_km to z_to_km.  z_from must be a multiple of L; (z_to - z_from)/L
 * whole; no amplifier strictly inside an interval (else MPA_ERR_GRID).
 * The lumped gain of an amplifier at an interval end is applied after
 * step 7.  Asynchronous on `stream`. */
MPA_API int mpa_propagate(mpa_plan* plan, void* field, double z_from_km, double z_to_km, mpa_stream stream);

/* One interval of the MPA without step 7: from the spectrum psi0 (N
 * complex128, natural frequency order, = A_hat(z0)) compute
 * psi^{(n_iter)} at node M (complex128) for the interval starting at z0_km
 * (a multiple of L).  Exposed for step-level parity checks. */
MPA_API int mpa_interval(mpa_plan* plan, const void* psi0, void* psiM, double z0_km, mpa_stream stream);

/* Picks the four-step split N = N1 x N2 of the plan's transforms by timing:
 * one interval (MPA steps 2-7) is run on the GPU for every admissible
 * column length N2 = 2^l (l within 3 of log2(N)/2, both passes supported,
 * and the reverse-mode tiling kept valid) and the fastest is kept.
 * Overwrites the plan's working buffers (call it before propagating) and
 * synchronises the stream.  *log2_n2 (may be NULL) receives the choice.
 * The split changes only the order of FP32 rounding, not the method.
 * Level-schedule plans only (a WAVEFRONT plan is left unchanged).  The paper
 * has no counterpart; this is the library's own tuning. */
MPA_API int mpa_plan_autotune(mpa_plan* plan, mpa_stream stream, int32_t* log2_n2);

/* Sets the split to column length 2^log2_n2 without timing (e.g. a value an
 * earlier mpa_plan_autotune chose).  MPA_ERR_UNSUPPORTED_N if the passes or
 * the reverse-mode tiling do not support it; a WAVEFRONT plan accepts only
 * its current split.  log2_n2 = 0 selects the on-chip node transform where N
 * allows it (N <= 2^16 FP32, 2^13 FP64): MPA steps 2-4 and the weight of
 * Eq. (6) for a node in one kernel, the spectrum held in shared memory (one
 * CTA up to 2^14 FP32 / 2^13 FP64; for FP32 2^15 and 2^16 a cluster of 2 or
 * 4 CTAs exchanging through distributed shared memory).  It is the default
 * of FP32 plans up to 2^14; mpa_plan_autotune tries it first and reports it
 * as 0.
 * Host-only. */
MPA_API int mpa_plan_set_split(mpa_plan* plan, int32_t log2_n2);

/* Run-time checks of the propagations since the last call (synchronises the
 * stream; clears the flags):
 *   MPA_ERR_NONFINITE  an interval result (step 7) held a NaN/Inf;
 *   MPA_ERR_DIVERGED   the Picard iteration of the text before MPA step 1
 *                      did not contract in some interval: the relative
 *                      increment at node M, ||psi^{(n+1)}_M - psi^{(n)}_M|| /
 *                      ||psi^{(n+1)}_M|| (all frequencies), failed to shrink
 *                      from one iteration to the next while above 1e-5 (the
 *                      rounding floor of the node-M sums).  The iteration
 *                      converges when L << z_nl (the paragraph after Eq. (2));
 *                      this is what a too long interval or too strong
 *                      nonlinearity produces.  Needs n_iter >= 2 and the
 *                      level schedule (the wavefront schedule reports only
 *                      MPA_ERR_NONFINITE);
 *   MPA_ERR_TIMEOUT    a bounded wait of the staged row pass (four-step
 *                      rows of 2^9 .. 2^13 points) ran out: the results
 *                      are incomplete (not expected in normal operation).
 * MPA_ERR_NONFINITE takes precedence; else MPA_OK. */
MPA_API int mpa_plan_status(mpa_plan* plan, mpa_stream stream);

/* The largest contraction factor rel_n / rel_{n-1} of the Picard increments
 * (as defined at mpa_plan_status) over all intervals and iterations
 * n >= 1 since the last call, into *worst (0 if none was measured);
 * synchronises the stream and resets the value.  Well below 1 in the
 * weakly nonlinear regime (about L / z_nl); >= 1 means no contraction. */
MPA_API int mpa_plan_contraction(mpa_plan* plan, mpa_stream stream, double* worst);

/* Scale check of the assumptions after Eq. (2): weak nonlinearity
 * z_nl >> z_disp, and an interval L well below z_nl (the Picard iteration
 * contracts by about L / z_nl) and L <~ z_disp.  With the typical peak power
 * P (W) and pulse width tau (ps) of the field:
 *   z_nl = 1 / (sigma_max P)          sigma_max: largest sigma of the map
 *   z_disp = tau^2 / <|beta2|>        <|beta2|>: length-weighted mean over a period
 * (km; written when the pointers are not NULL).  *flags (may be NULL)
 * receives MPA_SCALE_* bits.  Returns MPA_ERR_SCALES when z_nl <= z_disp or
 * L >= z_nl; MPA_SCALE_L_ABOVE_ZDISP alone (a soft condition of the paper)
 * still returns MPA_OK.  Host only. */
enum { MPA_SCALE_STRONG_NONLINEARITY = 1, MPA_SCALE_L_ABOVE_ZNL = 2, MPA_SCALE_L_ABOVE_ZDISP = 4 };
MPA_API int mpa_plan_check_scales(const mpa_plan* plan, double peak_power_W, double pulse_width_ps,
                                  double* z_nl_km, double* z_disp_km, int32_t* flags);

MPA_API void mpa_plan_destroy(mpa_plan* plan);

/* ---- Reverse mode (gradients of a real loss) ----------------------------
 * The reverse mode of the discrete method that mpa_propagate runs (MPA steps
 * 2-7 with Eq. (6), walked backwards), for a real loss l of the output field
 * A_out.  A gradient of a complex quantity x is dl/dRe x + i dl/dIm x (the
 * convention of torch's complex autograd).  Parameters are those of the
 * physical segments: segment s of period p is index p n_segments + s, for
 * n_periods x n_segments values (mpa_plan_n_segments).  The paper has no
 * adjoint; this is the gradient of its method (beta2 and sigma enter through
 * the phases beta(w, z_j) and sigma(z_j) of Eq. (6) and step 7).
 *
 * Memory: a checkpoint of A_hat (complex128) at every interval start, then,
 * for one interval at a time, psi^{(n)}, A^{(n)}(t) and V^{(n)} of every
 * level and the running gradient (3 n_iter buffers of (M+1) N samples in
 * all) and a few buffers of N samples.  Level-schedule
 * plans only (MPA_SCHEDULE_WAVEFRONT plans are rejected with
 * MPA_ERR_INVALID_ARG), and N >= 2^13 (MPA_ERR_UNSUPPORTED_N).
 * The workspace is caller-owned device memory, 256-byte aligned. */
MPA_API int mpa_plan_n_segments(const mpa_plan* plan, int32_t* n);
MPA_API int mpa_adjoint_workspace_size(const mpa_plan* plan, double z_from_km, double z_to_km, size_t* bytes);

/* mpa_propagate that also stores the checkpoints of [z_from, z_to] in the
 * adjoint workspace (for a later mpa_adjoint with field_in = NULL). */
MPA_API int mpa_propagate_checkpointed(mpa_plan* plan, void* field, double z_from_km, double z_to_km,
                                       void* adj_workspace, size_t adj_bytes, mpa_stream stream);

/* Gradients of l through mpa_propagate over [z_from, z_to].
 *   field_in   the input field A(z_from) (device, precision's complex type), or
 *              NULL: reuse the checkpoints of the last mpa_propagate_checkpointed
 *              over the same range with the same workspace.
 *   grad_out   dl/dA_out (device, N samples); not modified.
 *   grad_in    receives dl/dA_in (device, N samples).
 *   grad_sigma, grad_beta2   HOST arrays of n_periods x n_segments doubles
 *              (either may be NULL); when any is given the call synchronises
 *              the stream before returning.
 * Errors: MPA_ERR_GRID as mpa_propagate; MPA_ERR_WORKSPACE if adj_bytes is
 * below mpa_adjoint_workspace_size or the pointer is misaligned. */
MPA_API int mpa_adjoint(mpa_plan* plan, const void* field_in, const void* grad_out, void* grad_in,
                        double z_from_km, double z_to_km, void* adj_workspace, size_t adj_bytes,
                        double* grad_sigma, double* grad_beta2, mpa_stream stream);

/* Many independent links propagated together (no counterpart in the paper;
 * the batching of independent problems of the MPA node transforms).  Each
 * link has its own fiber map, N, window and length z_to (from z = 0, a
 * multiple of L_km); all share the discretisation L_km, M, n_iter and the
 * precision.  Links with equal N are batched into the same launches (each
 * with its own node constants); groups of different N run as parallel
 * branches of one CUDA graph.  Field pointers are fixed at creation (the
 * graph captures them); fields are updated in place, as by mpa_propagate. */
typedef struct {
    mpa_fiber_map map;  /* copied at creation */
    int64_t N;
    double T_ps;
    double z_to_km;     /* propagation 0 -> z_to_km */
    void* field;        /* device, N samples of the batch precision's complex type */
} mpa_link;

typedef struct mpa_batch mpa_batch;

/* L_km and M obey the limits of mpa_plan_params; each link has at most
 * 2^31 - 1 intervals (MPA_ERR_GRID). */
MPA_API int mpa_batch_create(const mpa_link* links, int32_t n_links, double L_km, int32_t M, int32_t n_iter,
                             int32_t precision, mpa_batch** out);
MPA_API int mpa_batch_workspace_size(const mpa_batch* batch, size_t* bytes);
/* Attaches caller-owned device workspace and uploads the node tables
 * (synchronous); a previously captured graph is discarded. */
MPA_API int mpa_batch_set_workspace(mpa_batch* batch, void* workspace, size_t bytes);
/* mpa_plan_autotune for every N group of the batch: times the group's first
 * interval for each admissible four-step split and keeps the fastest.
 * Overwrites the batch's working buffers (call it before propagating; the
 * fields are not touched), drops a captured graph, synchronises. */
MPA_API int mpa_batch_autotune(mpa_batch* batch, mpa_stream stream);
/* Propagates every link.  use_graph != 0: the first such call runs the
 * launches directly and captures them into a CUDA graph (one parallel
 * branch per N group, on library-owned streams joined to `stream`); later
 * calls replay the graph on `stream`.  Do not call it while `stream` is
 * being captured by the caller. */
MPA_API int mpa_batch_propagate(mpa_batch* batch, int32_t use_graph, mpa_stream stream);
/* mpa_plan_status for all links of the batch: MPA_ERR_TIMEOUT (a wait of
 * a persistent kernel ran out: the results are incomplete), else
 * MPA_ERR_NONFINITE or MPA_ERR_DIVERGED if any link produced it since the
 * last call (synchronises the stream, clears the flags), else MPA_OK. */
MPA_API int mpa_batch_status(mpa_batch* batch, mpa_stream stream);

/* Groups of FP32 links on the single-CTA on-chip node transform (N <= 2^14)
 * can run every interval and Picard iteration of all their links in ONE
 * persistent launch: a work queue over (link, interval, iteration, node
 * block) and (link, interval, iteration, frequency block), where the CTA
 * that finishes a link's phase enqueues the next (the scan after the nodes,
 * the next iteration or interval after the scan), so links advance
 * independently.  The only waits are on queue slots, bounded by the wait
 * limit (default 2^24 polls, about 2 s); a wait that runs out ends the
 * kernel with MPA_ERR_TIMEOUT in mpa_batch_status.  mpa_batch_autotune
 * chooses per group between it and per-pass launches; this call sets it
 * for every eligible group (on != 0) or none.  Both drop a captured graph.
 * The paper has no counterpart (the batching of independent problems). */
MPA_API int mpa_batch_set_persistent(mpa_batch* batch, int32_t on);
/* The wait limit (polls >= 0) of the batch's persistent kernels: the work
 * queue above, and the staged row pass of four-step node transforms with
 * rows of 2^9 .. 2^13 points, whose waits on its staging copies are bounded
 * the same way (plans use 2^22 polls).  polls = 0 makes every such wait run
 * out at once (for tests of MPA_ERR_TIMEOUT).  Drops a captured graph. */
MPA_API int mpa_batch_set_wait_limit(mpa_batch* batch, int64_t polls);
MPA_API void mpa_batch_destroy(mpa_batch* batch);

/* Symmetric split-step of Eq. (4) on the GPU: half linear step, then
 * (nonlinear phase rotation exp(i sigma |A|^2 dz), linear step) repeated,
 * the last linear step halved.  Linear steps are exact Fourier multipliers
 * exp(i beta(w; za, zb) + int G) (amplifier gains included); the nonlinear
 * step uses int sigma over the step.  (z_to - z_from)/dz must be whole.
 * The field (precision's complex type) is updated in place. */
MPA_API int ss_workspace_size(int64_t N, int32_t precision, size_t* bytes);
MPA_API int ss_propagate(const mpa_fiber_map* map, int64_t N, double T_ps, double dz_km, int32_t precision,
                 void* field, double z_from_km, double z_to_km, void* workspace, size_t ws_bytes,
                 mpa_stream stream);

/* Reverse mode of ss_propagate (the split-step of Eq. (4)) for a real loss,
 * in the conventions of mpa_adjoint: given the input field and grad_out =
 * dl/dA_out (device, N samples each, the precision's complex type), writes
 * dl/dA_in to grad_in and, when given, the per-physical-segment dl/dsigma
 * and dl/dbeta2 to HOST arrays of n_periods x n_segments doubles (the call
 * then synchronises the stream).  The forward pass is repeated with a
 * checkpoint every ckpt_steps steps (<= 0: about sqrt of the step count);
 * each checkpoint segment is recomputed with the field before every
 * nonlinear step and the spectrum after every linear step kept.  Memory:
 * (checkpoints + 2 ckpt_steps + 3) N samples.  N >= 2^13.  The paper has
 * no adjoint; this is the gradient of Eq. (4) as ss_propagate computes it. */
MPA_API int ss_adjoint_workspace_size(const mpa_fiber_map* map, int64_t N, int32_t precision, double dz_km,
                                      double z_from_km, double z_to_km, int32_t ckpt_steps, size_t* bytes);
MPA_API int ss_adjoint(const mpa_fiber_map* map, int64_t N, double T_ps, double dz_km, int32_t precision,
                       const void* field_in, const void* grad_out, void* grad_in, double z_from_km, double z_to_km,
                       int32_t ckpt_steps, void* workspace, size_t ws_bytes, double* grad_sigma, double* grad_beta2,
                       mpa_stream stream);

/* Discrete Fourier transform of N values in place, in the convention above:
 * sign = +1: F (no scaling), sign = -1: F^-1 (scaled by 1/N).  The MPA uses
 * these transforms in steps 3 and 4.  Workspace: ss_workspace_size bytes. */
MPA_API int mpa_fft(int64_t N, int32_t precision, int32_t sign, void* data, void* workspace, size_t ws_bytes,
            mpa_stream stream);

/* Size limit of mpa_fft_noalloc: N times the element size (8 or 16 bytes)
 * may not exceed this many bytes (N <= 2^20 in FP32, 2^19 in FP64). */
#define MPA_FFT_NOALLOC_MAX_BYTES (8u << 20)

/* mpa_fft for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a library convenience.  A plugin inside a host
 * application that owns all device memory through its own pool, or a
 * latency-critical loop that must not stall on cudaMalloc, may have no
 * workspace to pass: this entry point takes only `data` (N samples of the
 * precision's complex type, transformed in place exactly as mpa_fft does)
 * and uses a scratch array compiled into the library, which every GPU that
 * loads the library holds (MPA_FFT_NOALLOC_MAX_BYTES) until the process
 * exits.  It calls no cudaMalloc, cudaFree or allocating routine.
 * Each call made outside stream capture looks up the array's device address
 * with the current device (so a device reset that recreates the context is
 * picked up); a call under stream capture reuses the address of the last
 * uncaptured call on that device, so make one call on each device before any
 * stream capture (without one: MPA_ERR_CUDA).
 * All calls share the one array, so calls that overlap on the GPU race:
 * order them on one stream or synchronise between them.  Nothing in the
 * array needs to start at zero (each call overwrites what it reads).
 * Errors: MPA_ERR_WORKSPACE when N times the element size exceeds
 * MPA_FFT_NOALLOC_MAX_BYTES; otherwise as mpa_fft. */
MPA_API int mpa_fft_noalloc(int64_t N, int32_t precision, int32_t sign, void* data, mpa_stream stream);

/* Human-readable status; the last CUDA error string for MPA_ERR_CUDA. */
MPA_API const char* mpa_status_string(int status);
MPA_API const char* mpa_last_cuda_error(void);

/* Number of this library's kernels launched since load (all threads). */
MPA_API int64_t mpa_kernel_launches(void);

/* Fault injection for tests of the error paths (tooling; the paper has no
 * counterpart).  after_launches >= 0 arms it: the kernel launch that many
 * launches from now (0: the next one) is not made, and the entry point that
 * attempted it returns MPA_ERR_CUDA with cuda_error (a cudaError_t value,
 * nonzero) as mpa_last_cuda_error.  It fires once, then disarms;
 * after_launches < 0 disarms.  Process-wide, shared by all threads.  No
 * GPU is touched: the launch is skipped on the host. */
MPA_API int mpa_debug_fail_launch(int64_t after_launches, int32_t cuda_error);

/* Measured fused multiply-add throughput of the current device in FP64
 * (MPA_FP64) or FP32 (MPA_FP32), in flop/s (2 per FMA), into *flops_per_s:
 * the ALU roofline of the FP64 split-step comparator (tooling; the paper has
 * no counterpart).  Runs a short kernel of independent FMA chains on
 * `stream` (tens of ms) and synchronises; allocates nothing. */
MPA_API int mpa_alu_peak(int32_t precision, double* flops_per_s, mpa_stream stream);

/* Launch timing (tooling): with enable != 0 every subsequent launch of a
 * column pass, row pass or scan is bracketed by CUDA events on its stream
 * (totals reset); mpa_profile_read synchronises on the recorded events and
 * returns, for kernel kind `kind` (0 .. mpa_profile_kind_name() == NULL),
 * the summed device time in ms, the number of launches and the summed
 * algorithmic bytes (each element a launch must read or write, counted
 * once). */
MPA_API void mpa_profile(int enable);
MPA_API int mpa_profile_read(int kind, double* total_ms, int64_t* launches, double* bytes);
MPA_API const char* mpa_profile_kind_name(int kind);

/* Per-call timing (tooling): while mpa_profile is enabled, each call of
 * mpa_propagate, mpa_interval, ss_propagate, mpa_propagate_checkpointed,
 * mpa_adjoint, ss_adjoint, mpa_batch_propagate and mpa_fft made on a
 * stream that is not capturing is bracketed by CUDA events on its stream
 * (an entry point called from inside another is not timed separately).
 * mpa_last_timing waits for the end event of the most recent timed call
 * (any thread) and writes its device time in ms to *ms and the entry
 * point's name (static storage) to *entry (may be NULL).
 * MPA_ERR_INVALID_ARG if ms is NULL or no call was timed since
 * mpa_profile(1); MPA_ERR_CUDA if an event failed. */
MPA_API int mpa_last_timing(double* ms, const char** entry);

/* Debug build (tooling; the library compiled with MPA_DEBUG_BOUNDS=1, a
 * separate libmpa_debug.so): every global access of the MPA passes, the
 * scan and the on-chip node transform of plans and batches (not of the
 * persistent batch kernel, the transforms, the split-step or the reverse
 * mode) is checked against the plan's or batch's workspace; an access
 * outside it is skipped (a load reads zero) and reported as MPA_ERR_BOUNDS
 * by mpa_plan_status / mpa_batch_status, instead of touching memory.
 * mpa_debug_bounds_checked returns 1 in such a build, 0 otherwise.
 * mpa_debug_set_bounds narrows a plan's checked range to [workspace + lo,
 * workspace + hi) (lo = hi = 0: the whole workspace), for tests that make
 * the check fire without any access leaving the workspace; no effect in
 * release builds.  MPA_ERR_INVALID_ARG for lo > hi or hi beyond the
 * workspace, MPA_ERR_WORKSPACE without one. */
MPA_API int32_t mpa_debug_bounds_checked(void);
MPA_API int mpa_debug_set_bounds(mpa_plan* plan, size_t lo, size_t hi);

#ifdef __cplusplus
}
#endif
#endif /* MPA_H */
