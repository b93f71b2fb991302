// Batched MPA propagation of many independent links (mpa_batch_*).
//
// Links with the same N form a group; a group's links are stored link-major
// (node spectra, FP64 states, working copies of psi_0) and every pass of
// the level-synchronous interval covers all of the group's links that are
// still propagating in one launch, each link with its own node constants
// (its own fiber map, window and interval start).  Links are ordered by
// length, so the links still running at interval q are a prefix.  Groups are
// independent: captured into one CUDA graph they become parallel branches,
// so small-N groups fill the GPU together.
#include <algorithm>
#include <memory>
#include <new>

#include "host.h"
#include "kp.cuh"

using namespace mpa;
using namespace mpa::host;

namespace {

struct Link {
    HostMap map;
    long long N;
    double T, z_to;
    void* field;
    long n_int;
    int n_types;
    size_t node_base;  // offset of its node table in the group's table
};

struct Group {
    Split sp;
    std::vector<int> links;        // batch link indices, longest first
    std::vector<NodeC> nodes;      // concatenated per-link tables
    std::vector<int> loff;         // [q][active link]
    std::vector<double> gain;      // [q][active link]
    std::vector<int> active;       // links running at interval q
    long n_int = 0;
    size_t off_psi = 0, off_state = 0, off_psi0c = 0, off_nodes = 0, off_loff = 0, off_gain = 0, off_err = 0;
    size_t off_conv = 0, off_dprev = 0;  // Picard increment check: ConvState and D at node M per link
    bool has_work = false;               // second set of node buffers (tile layout of the staged column passes)
    size_t off_work = 0;
    // persistent work-queue kernel (FP32 groups on the single-CTA on-chip transform)
    bool persistent = false;
    unsigned int q_cap = 0;
    size_t off_qtask = 0, off_qseq = 0, off_ctr = 0, off_nint = 0;
    std::vector<int> link_nint;  // intervals per link (group order)
};

// Whether the group can run on the persistent kernel: FP32 spectra that fit
// one CTA, the on-chip node transform chosen.
bool persistent_ok(const Group& g, int prec) {
    return prec == MPA_FP32 && g.sp.onchip && g.sp.N <= (1ll << 14);
}

Monitor group_monitor(unsigned char* ws, size_t ws_bytes, const Group& g, long long spin_limit) {
    Monitor m{};
    m.spin_limit = spin_limit;
    m.dbg = DbgRange{reinterpret_cast<const char*>(ws), reinterpret_cast<const char*>(ws + ws_bytes),
                     reinterpret_cast<unsigned int*>(ws + g.off_err)};
    m.err = reinterpret_cast<unsigned int*>(ws + g.off_err);
    m.conv = reinterpret_cast<ConvState*>(ws + g.off_conv);
    m.dprev = reinterpret_cast<float2*>(ws + g.off_dprev);
    return m;
}

}  // namespace

struct mpa_batch {
    double L;
    int M, n_iter, prec;
    long long spin_limit = 1ll << 24;  // polls of a persistent-kernel wait (about 2 s)
    size_t csize;
    std::vector<Link> links;
    std::vector<Group> groups;
    size_t ws_need = 0;
    size_t ws_bytes = 0;
    unsigned char* ws = nullptr;
    cudaGraphExec_t graph = nullptr;
    long long graph_kernels = 0;  // kernel nodes per replay
    cudaStream_t cap = nullptr;  // capture origin
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> ev;
};

namespace {

int link_type(const Link& k, double L, double z0, int* t) {
    if (k.n_types == 1) {
        *t = 0;
        return MPA_OK;
    }
    const double u = z0 - std::floor(z0 / k.map.period + 1e-12) * k.map.period;
    double r;
    if (!whole(u / L, &r)) return MPA_ERR_GRID;
    long q = (long)r % k.n_types;
    if (q < 0) q += k.n_types;
    *t = (int)q;
    return MPA_OK;
}

// All intervals (at most q_limit per link) of a group on the persistent
// kernel, from the states and working copies in the workspace.
int run_persistent(mpa_batch* b, Group& g, int q_limit, cudaStream_t st) {
    const Split& s = g.sp;
    const int n = (int)g.links.size();
    KPParams k{};
    k.psi = reinterpret_cast<float2*>(b->ws + g.off_psi);
    k.psi0c = reinterpret_cast<float2*>(b->ws + g.off_psi0c);
    k.state = reinterpret_cast<double2*>(b->ws + g.off_state);
    k.nodes = reinterpret_cast<const NodeC*>(b->ws + g.off_nodes);
    k.loff = reinterpret_cast<const int*>(b->ws + g.off_loff);
    k.gain = reinterpret_cast<const double*>(b->ws + g.off_gain);
    k.conv = reinterpret_cast<ConvState*>(b->ws + g.off_conv);
    k.dprev = reinterpret_cast<float2*>(b->ws + g.off_dprev);
    k.err = reinterpret_cast<unsigned int*>(b->ws + g.off_err);
    k.n_int = reinterpret_cast<const int*>(b->ws + g.off_nint);
    k.N = s.N;
    k.M = b->M;
    k.n_iter = b->n_iter;
    k.n_links = n;
    k.nb = (b->M + 1 + KN_TILE_ROWS(s.logN) - 1) / KN_TILE_ROWS(s.logN);
    k.ns = (int)(s.N / KN_THREADS(s.logN));
    k.q_limit = q_limit;
    k.inv_n = (float)(1.0 / (double)s.N);
    k.floor_rel = kDivergenceFloor;
    k.q_task = reinterpret_cast<unsigned long long*>(b->ws + g.off_qtask);
    k.q_seq = reinterpret_cast<unsigned int*>(b->ws + g.off_qseq);
    k.q_cap = g.q_cap;
    k.ctr = reinterpret_cast<unsigned int*>(b->ws + g.off_ctr);
    k.spin_limit = b->spin_limit;
    MPA_TRY(kp_init_launch(k.q_seq, k.q_cap, k.ctr, 3 + n, st));
    MPA_TRY(kp_launch(s.logN, k, st));
    return MPA_OK;
}

template <typename T>
int run_group(mpa_batch* b, Group& g, cudaStream_t st) {
    const Split& s = g.sp;
    const long long N = s.N;
    const int M = b->M, n = (int)g.links.size();
    cx<T>* psi = reinterpret_cast<cx<T>*>(b->ws + g.off_psi);
    double2* state = reinterpret_cast<double2*>(b->ws + g.off_state);
    cx<T>* psi0c = reinterpret_cast<cx<T>*>(b->ws + g.off_psi0c);
    const NodeC* nodes = reinterpret_cast<const NodeC*>(b->ws + g.off_nodes);
    const int* loff = reinterpret_cast<const int*>(b->ws + g.off_loff);
    const double* gain = reinterpret_cast<const double*>(b->ws + g.off_gain);
    const Monitor mon = group_monitor(b->ws, b->ws_bytes, g, b->spin_limit);
    // a fresh increment check per propagation (a run that ended early, e.g.
    // on a timeout, must not leave a half-counted level behind)
    MPA_TRY(cudaMemsetAsync(mon.conv, 0, (size_t)n * sizeof(ConvState), st));
    // A_hat(0) = F[A] for every link (its node-0 buffer is the scratch)
    for (int i = 0; i < n; ++i) {
        cx<T>* scratch = psi + (long long)i * (M + 1) * N;
        int rc = fft_forward<T>(s, reinterpret_cast<const cx<T>*>(b->links[(size_t)g.links[(size_t)i]].field), scratch, st);
        if (rc) return rc;
        MPA_TRY(to_state_launch<T>(scratch, state + (long long)i * N, sizeof(T) == 4 ? psi0c + (long long)i * N : nullptr,
                                   N, st));
    }
    if (g.persistent && persistent_ok(g, b->prec)) {
        // every interval of every link in one launch
        int rc = run_persistent(b, g, 1 << 30, st);
        if (rc) return rc;
    } else {
        for (long q = 0; q < g.n_int; ++q) {
            int rc = mpa_levels<T>(s, M, b->n_iter, g.active[(size_t)q], psi,
                                   g.has_work ? reinterpret_cast<cx<T>*>(b->ws + g.off_work) : nullptr, psi0c, state,
                                   nodes, loff + (size_t)q * n, gain + (size_t)q * n, mon, 1, nullptr, st);
            if (rc) return rc;
        }
    }
    for (int i = 0; i < n; ++i) {
        cx<T>* scratch = psi + (long long)i * (M + 1) * N;
        MPA_TRY(from_state_launch<T>(state + (long long)i * N, scratch, N, st));
        int rc = fft_inverse<T>(s, scratch, reinterpret_cast<cx<T>*>(b->links[(size_t)g.links[(size_t)i]].field), st);
        if (rc) return rc;
    }
    return MPA_OK;
}

int run_all(mpa_batch* b, cudaStream_t origin, bool fork) {
    if (!fork) {
        for (auto& g : b->groups) {
            int rc = b->prec == MPA_FP32 ? run_group<float>(b, g, origin) : run_group<double>(b, g, origin);
            if (rc) return rc;
        }
        return MPA_OK;
    }
    // one branch per group, joined back into the origin stream
    const size_t G = b->groups.size();
    MPA_TRY(cudaEventRecord(b->ev[0], origin));
    for (size_t i = 0; i < G; ++i) {
        MPA_TRY(cudaStreamWaitEvent(b->branch[i], b->ev[0], 0));
        Group& g = b->groups[i];
        int rc = b->prec == MPA_FP32 ? run_group<float>(b, g, b->branch[i]) : run_group<double>(b, g, b->branch[i]);
        if (rc) return rc;
        MPA_TRY(cudaEventRecord(b->ev[i + 1], b->branch[i]));
        MPA_TRY(cudaStreamWaitEvent(origin, b->ev[i + 1], 0));
    }
    return MPA_OK;
}

void release_graph(mpa_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (auto s : b->branch) cudaStreamDestroy(s);
    b->branch.clear();
    for (auto e : b->ev) cudaEventDestroy(e);
    b->ev.clear();
    if (b->cap) cudaStreamDestroy(b->cap);
    b->cap = nullptr;
}

}  // namespace

extern "C" {

int mpa_batch_create(const mpa_link* links, int32_t n_links, double L_km, int32_t M, int32_t n_iter,
                     int32_t precision, mpa_batch** out) {
    return abi_call([&]() -> int {
        if (!links || n_links < 1 || !out || !(L_km > 0.0) || M < 1 || M > kMaxNodes || n_iter < 1)
            return MPA_ERR_INVALID_ARG;
        if (precision != MPA_FP32 && precision != MPA_FP64) return MPA_ERR_INVALID_ARG;
        *out = nullptr;
        std::unique_ptr<mpa_batch> b(new mpa_batch());  // released to *out on success
        b->L = L_km;
        b->M = M;
        b->n_iter = n_iter;
        b->prec = precision;
        b->csize = precision == MPA_FP32 ? sizeof(float2) : sizeof(double2);
        b->links.resize((size_t)n_links);
        auto fail = [](int rc) { return rc; };
        const double dz = L_km / M;
        for (int i = 0; i < n_links; ++i) {
            const mpa_link& in = links[i];
            Link& k = b->links[(size_t)i];
            int rc = k.map.init(&in.map);
            if (rc) return fail(rc);
            if (!in.field || !(in.T_ps > 0.0)) return fail(MPA_ERR_INVALID_ARG);
            Split sp;
            rc = split_n(in.N, precision, &sp);
            if (rc) return fail(rc);
            k.N = in.N;
            k.T = in.T_ps;
            k.z_to = in.z_to_km;
            k.field = in.field;
            double r;
            if (!(in.z_to_km > 0.0) || in.z_to_km > k.map.length * (1 + 1e-12) + 1e-9 ||
                !whole(in.z_to_km / L_km, &r) || r > kMaxIntervals)
                return fail(MPA_ERR_GRID);
            k.n_int = (long)r;
            if (whole(k.map.period / L_km, &r) && r >= 1 && r <= kMaxIntervalTypes) k.n_types = (int)r;
            else if (whole(L_km / k.map.period, &r) && r >= 1) k.n_types = 1;
            else return fail(MPA_ERR_GRID);
            for (long q = 0; q < k.n_int; ++q) {
                const double z0 = L_km * (double)q;
                if (k.map.amp_inside(z0, z0 + L_km)) return fail(MPA_ERR_GRID);
            }
        }
        // groups by N, links longest first
        std::vector<int> order((size_t)n_links);
        for (int i = 0; i < n_links; ++i) order[(size_t)i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            const Link &x = b->links[(size_t)a], &y = b->links[(size_t)c];
            return x.N != y.N ? x.N < y.N : x.n_int > y.n_int;
        });
        for (int i : order) {
            const Link& k = b->links[(size_t)i];
            if (b->groups.empty() || b->groups.back().sp.N != k.N) {
                b->groups.emplace_back();
                split_n(k.N, precision, &b->groups.back().sp);
                // on-chip node transforms by default where an FP32 spectrum fits a CTA
                b->groups.back().sp.onchip = precision == MPA_FP32 && onchip_ok(k.N, MPA_FP32) && k.N <= (1ll << 14);
            }
            b->groups.back().links.push_back(i);
        }
        size_t off = 0;
        for (auto& g : b->groups) {
            const int n = (int)g.links.size();
            const size_t N = (size_t)g.sp.N;
            // node tables of every link (each interval start within its period),
            // allocated at once: a table too large for the host fails here
            size_t n_nodes = 0;
            for (int i = 0; i < n; ++i)
                n_nodes += (size_t)b->links[(size_t)g.links[(size_t)i]].n_types * ((size_t)M + 1);
            g.nodes.reserve(n_nodes);
            for (int i = 0; i < n; ++i) {
                Link& k = b->links[(size_t)g.links[(size_t)i]];
                k.node_base = g.nodes.size();
                for (int t = 0; t < k.n_types; ++t) {
                    const double u0 = L_km * t;
                    for (int j = 0; j <= M; ++j) {
                        const double zr = (j == M) ? L_km : dz * j;
                        NodeC c{};
                        phase_consts(k.map.integ(u0, u0 + zr, 1), k.map.integ(u0, u0 + zr, 2), k.T, &c);
                        c.pre = std::exp(k.map.G(u0, u0 + zr));
                        double sig;
                        if (j == 0) sig = k.map.side(u0, 3, +1);
                        else if (j == M) sig = k.map.side(u0 + zr, 3, -1);
                        else sig = 0.5 * (k.map.side(u0 + zr, 3, -1) + k.map.side(u0 + zr, 3, +1));
                        c.post = sig * dz / c.pre;
                        g.nodes.push_back(c);
                    }
                }
                g.n_int = std::max(g.n_int, k.n_int);
            }
            g.loff.assign((size_t)g.n_int * n, 0);
            g.gain.assign((size_t)g.n_int * n, 1.0);
            g.active.assign((size_t)g.n_int, 0);
            for (long q = 0; q < g.n_int; ++q) {
                int act = 0;
                for (int i = 0; i < n; ++i) {
                    const Link& k = b->links[(size_t)g.links[(size_t)i]];
                    if (k.n_int <= q) continue;
                    ++act;
                    const double z0 = L_km * (double)q;
                    int t;
                    if (link_type(k, L_km, z0, &t)) return fail(MPA_ERR_GRID);
                    g.loff[(size_t)q * n + i] = (int)(k.node_base + (size_t)t * (M + 1));
                    g.gain[(size_t)q * n + i] = std::exp((double)k.map.amps(z0, z0 + L_km) * k.map.z_a * k.map.gamma);
                }
                g.active[(size_t)q] = act;
            }
            g.off_psi = off;
            off = align256(off + (size_t)n * (M + 1) * N * b->csize);
            g.has_work = wants_work_buffers(N, precision);
            g.off_work = off;
            if (g.has_work) off = align256(off + (size_t)n * (M + 1) * N * b->csize);
            g.off_state = off;
            off = align256(off + (size_t)n * N * sizeof(double2));
            g.off_psi0c = precision == MPA_FP32 ? off : g.off_state;
            if (precision == MPA_FP32) off = align256(off + (size_t)n * N * sizeof(float2));
            g.off_nodes = off;
            off = align256(off + g.nodes.size() * sizeof(NodeC));
            g.off_loff = off;
            off = align256(off + g.loff.size() * sizeof(int));
            g.off_gain = off;
            off = align256(off + g.gain.size() * sizeof(double));
            g.off_err = off;
            off = align256(off + sizeof(unsigned int));
            g.off_conv = off;
            off = align256(off + (size_t)n * sizeof(ConvState));
            g.off_dprev = off;
            if (n_iter > 1) off = align256(off + (size_t)n * N * sizeof(float2));
            g.link_nint.resize((size_t)n);
            for (int i = 0; i < n; ++i) g.link_nint[(size_t)i] = (int)b->links[(size_t)g.links[(size_t)i]].n_int;
            if (precision == MPA_FP32 && g.sp.N <= (1ll << 14) && g.sp.N >= (1ll << KN_LOG_MIN)) {
                // queue of the persistent kernel: one phase of tasks per link, plus slack
                const long long rows = KN_TILE_ROWS(g.sp.logN), thr = KN_THREADS(g.sp.logN);
                const long long nb = (M + 1 + rows - 1) / rows, ns = (long long)N / thr;
                g.q_cap = (unsigned)((long long)n * (nb > ns ? nb : ns) + 4096);
                g.off_qtask = off;
                off = align256(off + (size_t)g.q_cap * sizeof(unsigned long long));
                g.off_qseq = off;
                off = align256(off + (size_t)g.q_cap * sizeof(unsigned int));
                g.off_ctr = off;
                off = align256(off + (size_t)(3 + n) * sizeof(unsigned int));
                g.off_nint = off;
                off = align256(off + (size_t)n * sizeof(int));
                g.persistent = g.sp.onchip;
            }
        }
        b->ws_need = off;
        *out = b.release();
        return MPA_OK;
    });
}

int mpa_batch_workspace_size(const mpa_batch* b, size_t* bytes) {
    if (!b || !bytes) return MPA_ERR_INVALID_ARG;
    *bytes = b->ws_need;
    return MPA_OK;
}

int mpa_batch_set_workspace(mpa_batch* b, void* ws, size_t bytes) {
    if (!b || !ws) return MPA_ERR_INVALID_ARG;
    if (bytes < b->ws_need || ((uintptr_t)ws & 255u) != 0) return MPA_ERR_WORKSPACE;
    release_graph(b);
    b->ws = reinterpret_cast<unsigned char*>(ws);
    b->ws_bytes = bytes;
    for (auto& g : b->groups) {
        MPA_TRY(cudaMemcpy(b->ws + g.off_nodes, g.nodes.data(), g.nodes.size() * sizeof(NodeC),
                           cudaMemcpyHostToDevice));
        MPA_TRY(cudaMemcpy(b->ws + g.off_loff, g.loff.data(), g.loff.size() * sizeof(int), cudaMemcpyHostToDevice));
        MPA_TRY(cudaMemcpy(b->ws + g.off_gain, g.gain.data(), g.gain.size() * sizeof(double), cudaMemcpyHostToDevice));
        MPA_TRY(cudaMemset(b->ws + g.off_err, 0, sizeof(unsigned int)));
        MPA_TRY(cudaMemset(b->ws + g.off_conv, 0, g.links.size() * sizeof(ConvState)));
        if (g.q_cap)
            MPA_TRY(cudaMemcpy(b->ws + g.off_nint, g.link_nint.data(), g.link_nint.size() * sizeof(int),
                               cudaMemcpyHostToDevice));
    }
    return MPA_OK;
}

int mpa_batch_status(mpa_batch* b, mpa_stream stream) {
    return abi_call([&]() -> int {
        if (!b) return MPA_ERR_INVALID_ARG;
        if (!b->ws) return MPA_ERR_WORKSPACE;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        std::vector<unsigned int> h(b->groups.size(), 0u);
        for (size_t i = 0; i < b->groups.size(); ++i)
            MPA_TRY(cudaMemcpyAsync(&h[i], b->ws + b->groups[i].off_err, sizeof(unsigned int),
                                    cudaMemcpyDeviceToHost, st));
        MPA_TRY(cudaStreamSynchronize(st));
        unsigned int all = 0u;
        for (size_t i = 0; i < b->groups.size(); ++i) {
            all |= h[i];
            MPA_TRY(cudaMemsetAsync(b->ws + b->groups[i].off_err, 0, sizeof(unsigned int), st));
        }
        return (all & ERR_TIMEOUT) ? MPA_ERR_TIMEOUT
             : (all & ERR_BOUNDS) ? MPA_ERR_BOUNDS
             : (all & ERR_NONFINITE) ? MPA_ERR_NONFINITE
             : (all & ERR_DIVERGED) ? MPA_ERR_DIVERGED
                                    : MPA_OK;
    });
}

int mpa_batch_set_persistent(mpa_batch* b, int32_t on) {
    if (!b) return MPA_ERR_INVALID_ARG;
    release_graph(b);  // the captured launches follow the old choice
    for (auto& g : b->groups) g.persistent = on != 0 && g.q_cap != 0;
    return MPA_OK;
}

int mpa_batch_set_wait_limit(mpa_batch* b, int64_t polls) {
    if (!b || polls < 0) return MPA_ERR_INVALID_ARG;
    b->spin_limit = polls;
    release_graph(b);  // the limit is a launch argument of the captured kernels
    return MPA_OK;
}

int mpa_batch_propagate(mpa_batch* b, int32_t use_graph, mpa_stream stream) {
    return abi_call([&]() -> int {
        EntryRange nv("mpa_batch_propagate", stream);
        if (!b) return MPA_ERR_INVALID_ARG;
        if (!b->ws) return MPA_ERR_WORKSPACE;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        if (!use_graph) return run_all(b, st, false);
        if (!b->graph) {
            // first call: run once directly (sets kernel attributes), then
            // capture the same launches, one parallel branch per N group
            int rc = run_all(b, st, false);
            if (rc) return rc;
            MPA_TRY(cudaStreamSynchronize(st));
            MPA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
            b->branch.resize(b->groups.size());
            for (auto& s : b->branch) MPA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            b->ev.resize(b->groups.size() + 1);
            for (auto& e : b->ev) MPA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            const bool prof = g_prof_on.exchange(false);
            MPA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            rc = run_all(b, b->cap, true);
            cudaGraph_t graph = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
            g_prof_on.store(prof);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            MPA_TRY(e);
            size_t nn = 0;
            cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> gn(nn);
            cudaGraphGetNodes(graph, gn.data(), &nn);
            b->graph_kernels = 0;
            for (auto& x : gn) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(x, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++b->graph_kernels;
            }
            const cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
            cudaGraphDestroy(graph);
            MPA_TRY(ei);
            // the launches recorded while capturing did not run
            g_launches.fetch_sub(b->graph_kernels, std::memory_order_relaxed);
            return MPA_OK;  // this call already propagated once
        }
        MPA_TRY(cudaGraphLaunch(b->graph, st));
        g_launches.fetch_add(b->graph_kernels, std::memory_order_relaxed);
        return MPA_OK;
    });
}

int mpa_batch_autotune(mpa_batch* b, mpa_stream stream) {
    if (!b) return MPA_ERR_INVALID_ARG;
    if (!b->ws) return MPA_ERR_WORKSPACE;
    release_graph(b);  // the captured launches use the old splits
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    MPA_TRY(cudaEventCreate(&e0));
    MPA_TRY(cudaEventCreate(&e1));
    int rc = MPA_OK;
    for (auto& g : b->groups) {
        const Split keep = g.sp;
        const int n = (int)g.links.size();
        const size_t N = (size_t)keep.N;
        Split best = keep;
        float best_ms = -1.f;
        // the on-chip node transform where N fits (first), then the four-step splits
        for (int l = keep.logN / 2 - 4; l <= keep.logN / 2 + 3 && rc == MPA_OK; ++l) {
            Split s;
            if (l == keep.logN / 2 - 4) {
                if (!onchip_ok(keep.N, b->prec) || split_n(keep.N, b->prec, &s) != MPA_OK) continue;
                s.onchip = true;
            } else if (split_with(keep.N, b->prec, l, &s) != MPA_OK) {
                continue;
            }
            g.sp = s;
            // the group's first interval on a zero field (timing does not depend on values)
            if (cudaMemsetAsync(b->ws + g.off_state, 0, (size_t)n * N * sizeof(double2), st) != cudaSuccess ||
                (b->prec == MPA_FP32 &&
                 cudaMemsetAsync(b->ws + g.off_psi0c, 0, (size_t)n * N * sizeof(float2), st) != cudaSuccess)) {
                rc = cuda_fail(cudaGetLastError());
                break;
            }
            float ms = 0.f;
            for (int rep = 0; rep < 2 && rc == MPA_OK; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) {
                    rc = MPA_ERR_CUDA;
                    break;
                }
                rc = b->prec == MPA_FP32
                         ? mpa_levels<float>(g.sp, b->M, b->n_iter, g.active[0],
                                             reinterpret_cast<float2*>(b->ws + g.off_psi),
                                             g.has_work ? reinterpret_cast<float2*>(b->ws + g.off_work) : nullptr,
                                             reinterpret_cast<float2*>(b->ws + g.off_psi0c),
                                             reinterpret_cast<double2*>(b->ws + g.off_state),
                                             reinterpret_cast<const NodeC*>(b->ws + g.off_nodes),
                                             reinterpret_cast<const int*>(b->ws + g.off_loff),
                                             reinterpret_cast<const double*>(b->ws + g.off_gain),
                                             group_monitor(b->ws, b->ws_bytes, g, b->spin_limit), 1, nullptr, st)
                         : mpa_levels<double>(g.sp, b->M, b->n_iter, g.active[0],
                                              reinterpret_cast<double2*>(b->ws + g.off_psi), nullptr,
                                              reinterpret_cast<double2*>(b->ws + g.off_psi0c),
                                              reinterpret_cast<double2*>(b->ws + g.off_state),
                                              reinterpret_cast<const NodeC*>(b->ws + g.off_nodes),
                                              reinterpret_cast<const int*>(b->ws + g.off_loff),
                                              reinterpret_cast<const double*>(b->ws + g.off_gain),
                                              group_monitor(b->ws, b->ws_bytes, g, b->spin_limit), 1, nullptr, st);
                if (rc == MPA_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = cuda_fail(cudaGetLastError());
            }
            if (rc == MPA_OK && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best = s;
            }
        }
        g.sp = rc == MPA_OK ? best : keep;
        if (rc == MPA_OK && g.q_cap && persistent_ok(g, b->prec)) {
            // the persistent kernel against the per-pass launches of the same
            // node transform, on the group's first interval
            float ms_p = 0.f;
            for (int rep = 0; rep < 2 && rc == MPA_OK; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) {
                    rc = cuda_fail(cudaGetLastError());
                    break;
                }
                rc = run_persistent(b, g, 1, st);
                if (rc == MPA_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms_p, e0, e1) != cudaSuccess))
                    rc = cuda_fail(cudaGetLastError());
            }
            g.persistent = rc == MPA_OK && ms_p < best_ms;
        } else {
            g.persistent = false;
        }
        if ((cudaMemsetAsync(b->ws + g.off_err, 0, sizeof(unsigned int), st) != cudaSuccess ||
             cudaMemsetAsync(b->ws + g.off_conv, 0, (size_t)n * sizeof(ConvState), st) != cudaSuccess) &&
            rc == MPA_OK)
            rc = cuda_fail(cudaGetLastError());
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

void mpa_batch_destroy(mpa_batch* b) {
    if (!b) return;
    release_graph(b);
    delete b;
}

}  // extern "C"
