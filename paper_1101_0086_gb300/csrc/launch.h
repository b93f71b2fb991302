// Host-side launchers of the kernels in kernels.cuh (one translation unit
// per kernel family and precision, compiled in parallel).
#pragma once

#include <atomic>

#include "kernels.cuh"

namespace mpa {

// Kernels launched by this library since load.
extern std::atomic<long long> g_launches;

// Host-side fault injection (mpa_debug_fail_launch): when armed, the launch
// gate of the n-th kernel launch from now returns the chosen error instead
// of launching, so the error paths of every entry point can be exercised
// without making a GPU fault.  Every launcher calls it before its launch.
extern std::atomic<long long> g_fail_countdown;  // < 0: disarmed
extern std::atomic<int> g_fail_code;
inline cudaError_t launch_gate() {
    if (g_fail_countdown.load(std::memory_order_relaxed) < 0) return cudaSuccess;
    const long long left = g_fail_countdown.fetch_sub(1, std::memory_order_acq_rel);
    if (left == 0) return static_cast<cudaError_t>(g_fail_code.load(std::memory_order_relaxed));
    if (left < 0) g_fail_countdown.store(-1, std::memory_order_relaxed);
    return cudaSuccess;
}

// One-time kernel attribute setup per device: cudaFuncSetAttribute applies
// to the current device only, so each launcher keeps one bit per device
// (devices 0..63; any higher device sets the attributes on every launch).
// Setting an attribute twice is harmless, so two threads racing on the first
// launch of a device need no lock.
struct AttrOnce {
    std::atomic<unsigned long long> mask{0};
};
template <class F> inline cudaError_t attrs_once(AttrOnce& once, F&& set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (once.mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = set();
    if (e == cudaSuccess && bit) once.mask.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Optional CUDA-event timing of every launch, by kernel kind (off by
// default; enabled through mpa_profile).
enum {
    PK_KC_MPA_PRE = 0, PK_KC_MPA_POST, PK_KC_SS, PK_KC_FFT, PK_KR_MPA, PK_KR_SS, PK_KR_FFT, PK_SCAN, PK_AUX,
    PK_KCW, PK_KC_ADJ, PK_KR_ADJ, PK_ADJ_AUX, PK_KN, PK_COUNT
};
extern std::atomic<bool> g_prof_on;
void prof_begin(cudaStream_t st);
void prof_end(int kind, cudaStream_t st, double bytes);
int prof_kc_kind(int mode);
// Per-call timer of the entry points (mpa_last_timing): while profiling is
// on, the outermost timed entry point of a thread records a CUDA event on
// its stream at construction and at destruction (not on a capturing stream).
class CallTimer {
  public:
    CallTimer(const char* name, cudaStream_t st);
    ~CallTimer();
    CallTimer(const CallTimer&) = delete;
    CallTimer& operator=(const CallTimer&) = delete;

  private:
    const char* name_;
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr;
};
void call_timing_reset();
// the most recent timed call: *have = false if there is none
cudaError_t call_timing_read(double* ms, const char** entry, bool* have);
int prof_kr_kind(int mode);
cudaError_t prof_read(int kind, double* ms, long long* n, double* bytes);
void prof_reset();

// Column/row lengths supported by the column pass (2^4..2^11) and the row
// pass (2^4..2^14 FP32, 2^4..2^13 FP64).
constexpr int KC_LOG_MIN = 4, KC_LOG_MAX = 11;
constexpr int KR_LOG_MIN = 4;
template <typename T> constexpr int kr_log_max() { return sizeof(T) == 4 ? 14 : 13; }

template <typename T> cudaError_t kc_launch(int mode, int logL, const KCParams<T>& p, cudaStream_t st);
template <typename T> cudaError_t kr_launch(int mode, int logL, const KRParams<T>& p, cudaStream_t st);
// whether kr_launch<float> takes the staged persistent row pass (krs.cuh)
bool kr_staged(int mode, int logL, const KRParams<float>& p);
// whether kc_launch<float> takes the staged persistent column pass (kcs.cuh)
bool kc_staged(int mode, int logL, const KCParams<float>& p);
// log2 of the columns per tile of the staged column pass for 2^logL-point
// columns (the tile layout's G), or -1 where there is none
int kcs_tile_log_cols(int logL);
// On-chip whole node transform for N = 2^logL, 2^8 <= N <= 2^kn_log_max:
// one CTA per node up to 2^14 (FP32) / 2^13 (FP64), a cluster of 2 or 4 CTAs
// over distributed shared memory for FP32 2^15 and 2^16 (knc_launch).
constexpr int KN_LOG_MIN = 8;
template <typename T> constexpr int kn_log_max() { return sizeof(T) == 4 ? 16 : 13; }
template <typename T> cudaError_t kn_launch(int logL, const KNParams<T>& p, cudaStream_t st);
cudaError_t knc_launch(int logL, const KNParams<float>& p, cudaStream_t st);
// Rows (nodes) per tile and threads per CTA of the FP32 on-chip transform
// for N = 2^logL <= 2^14 (KNGeom<float, N>: tiles of 8192 elements, 32 per thread).
#define KN_TILE_ROWS(logL) ((logL) >= 13 ? 1ll : (8192ll >> (logL)))
#define KN_THREADS(logL) ((logL) >= 14 ? 512ll : 256ll)
// Persistent batch kernel (kp.cuh): FP32, N = 2^logL <= 2^14, and its queue reset.
struct KPParams;
cudaError_t kp_launch(int logL, const KPParams& p, cudaStream_t st);
cudaError_t kp_init_launch(unsigned int* q_seq, unsigned int q_cap, unsigned int* ctr, int n_ctr, cudaStream_t st);
template <typename T> cudaError_t scan_launch(const ScanParams<T>& p, int links, cudaStream_t st);
template <typename T> cudaError_t transpose_launch(const cx<T>* in, cx<T>* out, long long R, long long C, cudaStream_t st);
template <typename T> cudaError_t to_state_launch(const cx<T>* in, double2* state, cx<T>* copy, long long N, cudaStream_t st);
template <typename T> cudaError_t from_state_launch(const double2* state, cx<T>* out, long long N, cudaStream_t st);

// Wavefront column pass (FP32): columns per tile for column length 2^logL,
// the launch, and the step-7 kernel that follows a wavefront interval.
int kcw_tile_cols(int logL);
cudaError_t kcw_launch(int logL, const KCWParams& p, cudaStream_t st);
cudaError_t reconstruct_launch(double2* state, float2* psi0c, const double2* D, const NodeC& nodeM, double gain,
                               long long N, unsigned int* err, double2* out, cudaStream_t st);

// Grid of a column pass over ncols columns of column length L.
template <typename T> long long kc_blocks(int logL, long long ncols);
template <typename T> long long kr_blocks(int logL, long long nrows);

}  // namespace mpa
