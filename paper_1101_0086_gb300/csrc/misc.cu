// Launchers of the scan, transpose and precision-conversion kernels, and the
// optional per-launch CUDA-event timer.
#include <mutex>
#include <vector>

#include "launch.h"
#include "mpa.h"

namespace mpa {

std::atomic<long long> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::atomic<long long> g_fail_countdown{-1};
std::atomic<int> g_fail_code{0};

namespace {
struct Prof {
    std::mutex mu;
    std::vector<cudaEvent_t> free_events;
    struct Pending {
        cudaEvent_t a, b;
        int kind;
        double bytes;
    };
    std::vector<Pending> pending;
    cudaEvent_t open = nullptr;
    double ms[PK_COUNT] = {};
    long long n[PK_COUNT] = {};
    double bytes[PK_COUNT] = {};
    cudaEvent_t get() {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    // fold finished intervals into the totals (synchronises on each end event)
    cudaError_t drain() {
        cudaError_t rc = cudaSuccess;
        for (auto& p : pending) {
            float t = 0.f;
            cudaError_t e = cudaEventSynchronize(p.b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
            if (e == cudaSuccess) {
                ms[p.kind] += t;
                n[p.kind] += 1;
                bytes[p.kind] += p.bytes;
            } else {
                rc = e;
            }
            free_events.push_back(p.a);
            free_events.push_back(p.b);
        }
        pending.clear();
        return rc;
    }
};
Prof& prof() {
    static Prof p;
    return p;
}
}  // namespace

void prof_begin(cudaStream_t st) {
    Prof& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    P.open = P.get();
    if (P.open) cudaEventRecord(P.open, st);
}

void prof_end(int kind, cudaStream_t st, double bytes) {
    Prof& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    if (!P.open) return;
    cudaEvent_t b = P.get();
    if (!b) return;
    cudaEventRecord(b, st);
    P.pending.push_back({P.open, b, kind, bytes});
    P.open = nullptr;
    if (P.pending.size() > 4096) P.drain();
}

namespace {
struct CallTiming {
    std::mutex mu;
    cudaEvent_t a = nullptr, b = nullptr;  // the most recent timed call
    const char* name = nullptr;
};
CallTiming& call_timing() {
    static CallTiming c;
    return c;
}
thread_local int t_call_depth = 0;
}  // namespace

CallTimer::CallTimer(const char* name, cudaStream_t st) : name_(name), st_(st) {
    if (t_call_depth++ > 0 || !g_prof_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();  // keep a failed query out of the launchers' error checks
        return;
    }
    if (cudaEventCreate(&a_) != cudaSuccess || cudaEventRecord(a_, st) != cudaSuccess) {
        cudaGetLastError();
        if (a_) cudaEventDestroy(a_);
        a_ = nullptr;
    }
}

CallTimer::~CallTimer() {
    --t_call_depth;
    if (!a_) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(b, st_) != cudaSuccess) {
        cudaGetLastError();
        if (b) cudaEventDestroy(b);
        cudaEventDestroy(a_);
        return;
    }
    CallTiming& C = call_timing();
    std::lock_guard<std::mutex> g(C.mu);
    if (C.a) cudaEventDestroy(C.a);
    if (C.b) cudaEventDestroy(C.b);
    C.a = a_;
    C.b = b;
    C.name = name_;
}

void call_timing_reset() {
    CallTiming& C = call_timing();
    std::lock_guard<std::mutex> g(C.mu);
    if (C.a) cudaEventDestroy(C.a);
    if (C.b) cudaEventDestroy(C.b);
    C.a = C.b = nullptr;
    C.name = nullptr;
}

cudaError_t call_timing_read(double* ms, const char** entry, bool* have) {
    CallTiming& C = call_timing();
    std::lock_guard<std::mutex> g(C.mu);
    *have = C.b != nullptr;
    if (!*have) return cudaSuccess;
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(C.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, C.a, C.b);
    if (e != cudaSuccess) return e;
    *ms = (double)t;
    if (entry) *entry = C.name;
    return cudaSuccess;
}

int prof_kc_kind(int mode) {
    return mode == KC_MPA_PRE ? PK_KC_MPA_PRE : mode == KC_MPA_POST ? PK_KC_MPA_POST
         : mode == KC_SS_STEP ? PK_KC_SS : PK_KC_FFT;
}
int prof_kr_kind(int mode) { return mode == KR_MPA ? PK_KR_MPA : mode == KR_SS ? PK_KR_SS : PK_KR_FFT; }

cudaError_t prof_read(int kind, double* ms, long long* n, double* bytes) {
    Prof& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    cudaError_t rc = P.drain();
    *ms = P.ms[kind];
    *n = P.n[kind];
    *bytes = P.bytes[kind];
    return rc;
}

void prof_reset() {
    Prof& P = prof();
    std::lock_guard<std::mutex> g(P.mu);
    P.drain();
    for (int k = 0; k < PK_COUNT; ++k) {
        P.ms[k] = 0.0;
        P.n[k] = 0;
        P.bytes[k] = 0.0;
    }
}

static unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T> cudaError_t scan_launch(const ScanParams<T>& p, int p_links, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    const bool pr = g_prof_on.load(std::memory_order_relaxed);
    if (pr) prof_begin(st);
    scan_kernel<T><<<dim3(blocks_for(p.N, 256), (unsigned)p_links), 256, 0, st>>>(p);
    if (pr) {
        const double cs = (double)sizeof(cx<T>), n = (double)p.N;
        double b = ((p.M + 1) * n * cs + n * cs) * p_links;  // V_0..V_M and psi_0
        if (p.mode == 0) b += p.M * n * cs * p_links;  // psi^{(n+1)}_1..M
        if (p.conv) b += ((p.level > 0 ? 8.0 : 0.0) + (p.level < p.n_iter - 1 ? 8.0 : 0.0)) * n * p_links;  // D at node M
        else b += (n * 16.0 + (p.mode == 1 ? n * (16.0 + cs) : n * 16.0)) * p_links;  // FP64 state in, result out
        prof_end(PK_SCAN, st, b);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t transpose_launch(const cx<T>* in, cx<T>* out, long long R, long long C, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    dim3 grid((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32));
    transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(in, out, R, C);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T>
cudaError_t to_state_launch(const cx<T>* in, double2* state, cx<T>* copy, long long N, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    to_state_kernel<T><<<blocks_for(N, 256), 256, 0, st>>>(in, state, copy, N);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template <typename T> cudaError_t from_state_launch(const double2* state, cx<T>* out, long long N, cudaStream_t st) {
    if (const cudaError_t eg = launch_gate()) return eg;
    from_state_kernel<T><<<blocks_for(N, 256), 256, 0, st>>>(state, out, N);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

template cudaError_t scan_launch<float>(const ScanParams<float>&, int, cudaStream_t);
template cudaError_t scan_launch<double>(const ScanParams<double>&, int, cudaStream_t);
template cudaError_t transpose_launch<float>(const float2*, float2*, long long, long long, cudaStream_t);
template cudaError_t transpose_launch<double>(const double2*, double2*, long long, long long, cudaStream_t);
template cudaError_t to_state_launch<float>(const float2*, double2*, float2*, long long, cudaStream_t);
template cudaError_t to_state_launch<double>(const double2*, double2*, double2*, long long, cudaStream_t);
template cudaError_t from_state_launch<float>(const double2*, float2*, long long, cudaStream_t);
template cudaError_t from_state_launch<double>(const double2*, double2*, long long, cudaStream_t);

}  // namespace mpa

extern "C" int mpa_debug_fail_launch(int64_t after_launches, int32_t cuda_error) {
    if (after_launches >= 0 && cuda_error == 0) return MPA_ERR_INVALID_ARG;
    mpa::g_fail_code.store(cuda_error, std::memory_order_relaxed);
    mpa::g_fail_countdown.store(after_launches < 0 ? -1 : (long long)after_launches, std::memory_order_release);
    return MPA_OK;
}
