// The single-link plan (host tables of the per-node constants of Eq. (6)
// and the workspace layout), shared by the forward schedule (plan.cu) and
// the reverse mode (adjoint.cu).
#pragma once

#include <vector>

#include "host.h"

struct mpa_plan {
    mpa::host::HostMap map;
    mpa::host::Split sp;
    double T, L;
    int M, n_iter, prec;
    int n_types;                // distinct interval starts within the DM period
    std::vector<mpa::NodeC> nodes;  // n_types x (M+1)
    size_t csize;               // bytes per complex sample
    size_t off_psi, off_state, off_psi0c, off_nodes, off_err, off_toff, off_gains, ws_need;
    size_t off_conv = 0, off_dprev = 0;  // Picard increment check (ConvState, D at node M)
    bool has_work = false;               // second set of node buffers (tile layout of the staged column passes)
    size_t off_work2 = 0;
    size_t dbg_lo = 0, dbg_hi = 0;       // debug build: checked range within the workspace (hi 0: all of it)
    // wavefront schedule (FP32): S = n_iter slots of B node buffers
    bool wf = false;
    int B = 0;
    size_t off_work = 0, off_y0 = 0, off_R = 0, off_C = 0, off_D = 0;
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
};

namespace mpa {
namespace host {

// The plan's run-time check words (error word, increment check).
Monitor monitor(const mpa_plan* p);

// MPA_ERR_TIMEOUT, MPA_ERR_BOUNDS, MPA_ERR_NONFINITE or MPA_ERR_DIVERGED for
// the bits of an error word (in that order of precedence: a timed-out wait
// or a skipped access leaves results incomplete).
inline int status_of_error_word(unsigned int h) {
    return (h & ERR_TIMEOUT) ? MPA_ERR_TIMEOUT
         : (h & ERR_BOUNDS) ? MPA_ERR_BOUNDS
         : (h & ERR_NONFINITE) ? MPA_ERR_NONFINITE
         : (h & ERR_DIVERGED) ? MPA_ERR_DIVERGED : MPA_OK;
}

// Index of the interval start z0 within the DM period (its node table).
int interval_type(const mpa_plan* p, double z0, int* t);

// One level-synchronous interval of the plan (MPA steps 2-7) on the plan's
// state; n_amp amplifiers end it; scan_mode as in ScanParams.
template <typename T>
int run_interval(mpa_plan* p, int type, long n_amp, int scan_mode, double2* out, cudaStream_t st);

}  // namespace host
}  // namespace mpa
