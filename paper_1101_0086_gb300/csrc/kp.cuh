// A persistent kernel that carries a group of equal-N links (N <= 2^14, FP32,
// the on-chip node transform) through every interval and Picard iteration
// of the MPA in one launch: a work queue over (link, interval, iteration,
// node block) and (link, interval, iteration, frequency block).
//
// Per link, an iteration is a node phase (MPA steps 2-4 and the weight of
// Eq. (6): nb tasks of G nodes, kn_tile) followed by a scan phase (step 5,
// and step 7 on the last iteration: ns tasks of NT frequencies, scan_freq).
// The CTA that finishes the last task of a phase (a per-link counter)
// pushes the next phase: the scan, the next iteration's nodes, the next
// interval's nodes, or marks the link done.  Links advance independently,
// so small links never wait for each other at level boundaries.
//
// The queue is a bounded ring of q_cap slots, each a task word and a
// sequence tag (the multi-producer multi-consumer ring with per-slot
// sequence numbers): slot i starts with tag i; a producer that took position
// pos (atomic on the tail) waits until the slot's tag is pos (its previous
// task was read), writes the task, fences and publishes the tag pos + 1; a
// consumer that took pos (atomic on the head) waits for the tag pos + 1,
// reads the task and frees the slot with the tag pos + q_cap.  These waits
// are the only ones in the kernel: a consumer's ends when its task arrives,
// when every link is done, or after spin_limit polls (about 128 ns each); a
// producer's after spin_limit polls too.  A wait that runs out records
// ERR_TIMEOUT in the error word and the CTA returns (the host reads it with
// mpa_batch_status).  q_cap covers every task that can be waiting in the
// queue (one phase per link), so producers do not wait in practice.  Data
// other CTAs wrote during the kernel is read through L2 (ld.global.cg).
#pragma once

#include "kernels.cuh"

namespace mpa {

struct KPParams {
    float2* psi;          // link l's node j at psi + (l (M+1) + j) N
    float2* psi0c;        // link l at + l N
    double2* state;       // link l at + l N
    const NodeC* nodes;
    const int* loff;      // [interval][link]
    const double* gain;   // [interval][link]
    ConvState* conv;      // per link
    float2* dprev;        // link l at + l N
    unsigned int* err;
    const int* n_int;     // intervals per link
    long long N;
    int M, n_iter, n_links, nb, ns, q_limit;
    float inv_n;
    double floor_rel;
    unsigned long long* q_task;
    unsigned int* q_seq;
    unsigned int q_cap;
    unsigned int* ctr;    // [0] head, [1] tail, [2] links done, [3 + l] tasks done in link l's phase
    long long spin_limit;
};

enum { KP_NODE = 0, KP_SCAN = 1 };

// task word: type (bit 63), iteration n (56-62), interval q (32-55), link (16-31), index (0-15)
__device__ __forceinline__ unsigned long long kp_word(unsigned type, unsigned n, unsigned q, unsigned l) {
    return ((unsigned long long)type << 63) | ((unsigned long long)(n & 127u) << 56) |
           ((unsigned long long)(q & 0xFFFFFFu) << 32) | ((unsigned long long)(l & 0xFFFFu) << 16);
}

// count tasks base | 0 .. count-1 onto the queue (one thread)
__device__ __forceinline__ void kp_push(const KPParams& p, unsigned long long base, int count) {
    const unsigned first = atomicAdd(p.ctr + 1, (unsigned)count);
    for (int i = 0; i < count; ++i) {
        const unsigned pos = first + (unsigned)i, slot = pos % p.q_cap;
        bool free = false;
        for (long long spins = 0; spins <= p.spin_limit; ++spins) {
            if (atomicAdd(p.q_seq + slot, 0u) == pos) {
                free = true;
                break;
            }
            __nanosleep(128);
        }
        if (!free) {
            atomicOr(p.err, ERR_TIMEOUT);
            return;
        }
        p.q_task[slot] = base | (unsigned long long)i;
        __threadfence();
        atomicExch(p.q_seq + slot, pos + 1u);
    }
}

template <int L>
__global__ void __launch_bounds__(KNGeom<float, L>::NT, 1) kp_kernel(const KPParams p) {
    typedef KNGeom<float, L> Gm;
    constexpr int NT = Gm::NT, G = Gm::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long s_task;
    __shared__ int s_stop;
    const int tid = threadIdx.x;
    unsigned* const done = p.ctr + 2;
    unsigned* const cnt = p.ctr + 3;
    const long long N = p.N, npl = p.M + 1;

    // the first iteration of every link's first interval
    if (blockIdx.x == 0 && tid == 0)
        for (int l = 0; l < p.n_links; ++l) kp_push(p, kp_word(KP_NODE, 0, 0, (unsigned)l), p.nb);

    for (;;) {
        if (tid == 0) {
            const unsigned pos = atomicAdd(p.ctr, 1u), slot = pos % p.q_cap;
            int stop = 0;
            for (long long spins = 0;; ++spins) {
                if (atomicAdd(p.q_seq + slot, 0u) == pos + 1u) {
                    __threadfence();
                    s_task = __ldcg(p.q_task + slot);
                    __threadfence();
                    atomicExch(p.q_seq + slot, pos + p.q_cap);  // free the slot for position pos + q_cap
                    break;
                }
                if (atomicAdd(done, 0u) >= (unsigned)p.n_links) {
                    stop = 1;
                    break;
                }
                if (spins >= p.spin_limit) {
                    atomicOr(p.err, ERR_TIMEOUT);
                    stop = 1;
                    break;
                }
                __nanosleep(128);
            }
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) return;
        const unsigned long long t = s_task;
        const unsigned type = (unsigned)(t >> 63), n = (unsigned)(t >> 56) & 127u;
        const unsigned q = (unsigned)(t >> 32) & 0xFFFFFFu, l = (unsigned)(t >> 16) & 0xFFFFu, idx = (unsigned)t & 0xFFFFu;
        const int* loff = p.loff + (long long)q * p.n_links + l;
        if (type == KP_NODE) {
            KNParams<float> k{};
            k.src = n == 0 ? p.psi0c + l * N : p.psi + l * npl * N;
            k.src_stride = n == 0 ? 0 : N;
            k.src0 = p.psi0c + l * N;
            k.dst = p.psi + l * npl * N;
            k.dst_stride = N;
            k.nrows = npl;
            k.npl = (int)npl;
            k.nodes = p.nodes;
            k.loff = loff;
            k.inv_n = p.inv_n;
            kn_tile<float, L, true>(k, (long long)idx * G, smem_raw);
        } else {
            ScanParams<float> s{};
            s.psi = p.psi + l * npl * N;
            s.N = N;
            s.M = p.M;
            s.psi0c = p.psi0c + l * N;
            s.state = p.state + l * N;
            s.psi0c_out = p.psi0c + l * N;
            s.mode = (int)n == p.n_iter - 1 ? 1 : 0;
            s.nodes = p.nodes;
            s.loff = loff;
            s.gain = p.gain + (long long)q * p.n_links + l;
            s.err = p.err;
            s.conv = p.conv + l;
            s.dprev = p.dprev + l * N;
            s.level = (int)n;
            s.n_iter = p.n_iter;
            s.floor_rel = p.floor_rel;
            scan_freq<float, true>(s, 0, (long long)idx * NT + tid, (unsigned)p.ns);
        }
        // this task's writes are visible before it is counted
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned need = type == KP_NODE ? (unsigned)p.nb : (unsigned)p.ns;
            if (atomicAdd(cnt + l, 1u) == need - 1u) {
                atomicExch(cnt + l, 0u);
                __threadfence();
                const int nq = p.n_int[l] < p.q_limit ? p.n_int[l] : p.q_limit;
                if (type == KP_NODE) kp_push(p, kp_word(KP_SCAN, n, q, l), p.ns);
                else if ((int)n + 1 < p.n_iter) kp_push(p, kp_word(KP_NODE, n + 1, q, l), p.nb);
                else if ((int)q + 1 < nq) kp_push(p, kp_word(KP_NODE, 0, q + 1, l), p.nb);
                else atomicAdd(done, 1u);
            }
        }
        __syncthreads();
    }
}

}  // namespace mpa
