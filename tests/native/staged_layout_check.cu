// Host-side check of the shared-memory layouts, copy ranges and the tile
// layout of the staged persistent passes (krs.cuh, kcs.cuh), for every
// supported length:
// the stage, the mbarriers, the node-constant slots, the twiddle tables and
// the two groups' exchange buffers and outer-factor tables are disjoint and
// fit the per-SM limit; every copy destination lies in the stage with the
// alignment its instruction needs; every stage element a thread reads was
// written by the tile's copies; and the per-group exchange slots the
// transforms address stay inside the group's buffer.  Prints the number of
// checks; exits non-zero on the first failure.
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>

#include "kcs.cuh"

using namespace mpa;

static long long g_checked = 0;

static void expect(bool ok, const char* what, int L) {
    ++g_checked;
    if (!ok) {
        std::printf("failed: %s (L = %d)\n", what, L);
        std::exit(1);
    }
}

struct Region {
    size_t lo, hi;
};
static void disjoint(const std::vector<Region>& r, size_t total, int L) {
    for (size_t i = 0; i < r.size(); ++i) {
        expect(r[i].lo <= r[i].hi && r[i].hi <= total, "region inside the block's shared memory", L);
        for (size_t j = i + 1; j < r.size(); ++j)
            expect(r[i].hi <= r[j].lo || r[j].hi <= r[i].lo, "regions disjoint", L);
    }
    expect(total <= 227u * 1024u, "at most 227 KB per block", L);
}

template <int L> void row_pass() {
    typedef KRSGeom<L> SG;
    typedef KRSTile<L> Gm;
    typedef Tiling<float, 1> P;
    const size_t C = sizeof(float2);
    std::vector<Region> r = {{0, SG::STAGE_BYTES}, {SG::BAR_OFF, SG::BAR_OFF + 16},
                             {SG::TW_OFF, SG::TW_OFF + (TwDims<L>::NLO + TwDims<L>::NHI) * C}};
    for (int g = 0; g < 2; ++g) {
        const size_t b = SG::GRP_OFF + g * SG::GRP_BYTES;
        r.push_back({b, b + (SG::S_ELEMS + (size_t)Gm::G * (Gm::OLO + Gm::OHI)) * C});
    }
    disjoint(r, SG::smem_bytes, L);
    expect(SG::BAR_OFF % 8 == 0 && SG::GRP_OFF % 16 == 0 && SG::GRP_BYTES % 16 == 0, "alignment", L);
    // the bulk copies: chunks of 16 KB covering nr rows (nr <= G), 16-byte sizes
    for (int nr = 1; nr <= Gm::G; ++nr) {
        const unsigned bytes = (unsigned)(nr * L * C);
        expect(bytes % 16 == 0 && bytes <= SG::STAGE_BYTES, "bulk copy size", L);
        for (unsigned o = 0; o < bytes; o += 16384) expect(o % 16 == 0, "bulk copy offset", L);
    }
    // stage reads of the first pass: element j + r L/R0 of row g
    typedef Xform<float, L, Gm::G, Gm::NT, P::RMAX, -1, LAYOUT_ROW, P::PSH, false, 1> XI;
    for (int tid = 0; tid < Gm::NT; ++tid)
        for (int q = 0; q < XI::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_ROW, L, Gm::G, XI::R0>(tid + q * Gm::NT, j, g);
            for (int rr = 0; rr < XI::R0; ++rr) expect(g * L + j + rr * (L / XI::R0) < Gm::TE, "stage read", L);
        }
    // exchange slots of both transforms stay in the group's buffer
    for (int i = 0; i < Gm::TE; ++i) expect((size_t)phys<P::PSH>(i) < SG::S_ELEMS, "exchange slot", L);
}

template <int L> void column_pass() {
    typedef KCSGeom<L> SG;
    typedef KCSTile<L> Gm;
    typedef Tiling<float> P;
    const size_t C = sizeof(float2);
    std::vector<Region> r = {{0, SG::STAGE_BYTES}, {SG::BAR_OFF, SG::BAR_OFF + 16},
                             {SG::NODE_OFF, SG::NODE_OFF + 4 * sizeof(NodeC)},
                             {SG::TW_OFF, SG::TW_OFF + (TwDims<L>::NLO + TwDims<L>::NHI) * C}};
    for (int g = 0; g < 2; ++g) {
        const size_t b = SG::GRP_OFF + g * SG::GRP_BYTES;
        r.push_back({b, b + (SG::S_ELEMS + (size_t)Gm::G * (Gm::OLO + Gm::OHI)) * C});
    }
    disjoint(r, SG::smem_bytes, L);
    expect(SG::NODE_OFF % 16 == 0 && sizeof(NodeC) % 16 == 0, "node slots take 16-byte copies", L);
    expect(Gm::TE == L * Gm::G, "tile of G whole columns", L);
    // the 16-byte copies of one tile: every stage byte written exactly once
    constexpr int CPR = Gm::G * (int)sizeof(float2) / 16, NCH = L * CPR;
    std::vector<int> hit(SG::STAGE_BYTES / 16, 0);
    for (int tid = 0; tid < Gm::NT; ++tid)
        for (int k = 0; k < NCH / Gm::NT; ++k) {
            const int id = tid + k * Gm::NT, row = id / CPR, ch = id % CPR;
            const size_t dst = (size_t)row * Gm::G * C + ch * 16;
            expect(dst % 16 == 0 && dst + 16 <= SG::STAGE_BYTES, "copy destination", L);
            ++hit[dst / 16];
        }
    for (int h : hit) expect(h == 1, "stage covered once", L);
    // stage reads of the first pass: element (row j + r L/R0, column g) at row G + g
    typedef Xform<float, L, Gm::G, Gm::NT, P::RMAX, -1, LAYOUT_COL, P::PSH, false, 1> XI;
    typedef Xform<float, L, Gm::G, Gm::NT, P::RMAX, +1, LAYOUT_COL, P::PSH, true, 1> XF;
    for (int tid = 0; tid < Gm::NT; ++tid) {
        for (int q = 0; q < XI::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, Gm::G, XI::R0>(tid + q * Gm::NT, j, g);
            for (int rr = 0; rr < XI::R0; ++rr) expect((j + rr * (L / XI::R0)) * Gm::G + g < Gm::TE, "stage read", L);
        }
        for (int q = 0; q < XF::Q0; ++q) {
            int j, g;
            bmap<LAYOUT_COL, L, Gm::G, XF::R0>(tid + q * Gm::NT, j, g);
            for (int rr = 0; rr < XF::R0; ++rr) expect((j + rr * (L / XF::R0)) * Gm::G + g < Gm::TE, "stage read", L);
        }
    }
    for (int i = 0; i < Gm::TE; ++i) expect((size_t)phys<P::PSH>(i) < SG::S_ELEMS, "exchange slot", L);
}

// The tile layout that the forward column pass writes, the scan keeps and
// the next inverse pass reads: for every node position, the forward pass's
// store address of (row k2, column k1) and the inverse pass's copy source of
// the same element coincide, and the scan maps that position back to
// k = k1 + N1 k2 (a bijection over the node).
template <int L> void tile_layout(int logN) {
    typedef KCSTile<L> Gm;
    constexpr int G = Gm::G;
    int logG = 0, logL = 0;
    while ((1 << logG) < G) ++logG;
    while ((1 << logL) < L) ++logL;
    const long long N = 1ll << logN, N1 = N >> logL;
    if (N1 % G != 0) return;
    KCParams<float> p{};
    float2* base = reinterpret_cast<float2*>(static_cast<uintptr_t>(1) << 40);  // address arithmetic only
    p.src = base;
    p.dst = base;
    p.src_stride = p.dst_stride = N;
    p.N = N;
    p.logN = logN;
    p.N1 = (int)N1;
    p.logN1 = logN - logL;
    p.npl = 3;
    p.ncols = 3 * N1;
    p.tiled_in = p.tiled_out = 1;
    std::vector<char> seen(N, 0);
    for (long long col0 = 0; col0 < p.ncols; col0 += G) {
        int l, jn;
        long long c, rs_in, rs_out;
        kcs_node(p, col0, l, jn, c);
        const float2* src = kcs_src<L, G>(p, l, jn, c, rs_in);
        float2* dst = kcs_dst<L, G>(p, l, jn, c, rs_out);
        expect(src == dst && rs_in == G && rs_out == G, "forward store and inverse copy agree", L);
        for (int k2 = 0; k2 < L; ++k2)
            for (int g = 0; g < G; ++g) {
                const long long i = (src + (long long)k2 * rs_in + g) - (base + (long long)jn * N);
                expect(i >= 0 && i < N, "position inside the node", L);
                expect(tile_to_natural(i, logG, logL, N) == (c + g) + N1 * k2, "scan maps the position back", L);
                if (jn == 1) {
                    expect(!seen[i], "bijection", L);
                    seen[i] = 1;
                }
            }
    }
}

int main() {
    tile_layout<256>(16);
    tile_layout<256>(20);
    tile_layout<512>(18);
    tile_layout<512>(20);
    tile_layout<1024>(20);
    tile_layout<1024>(24);
    tile_layout<2048>(22);
    tile_layout<2048>(24);
    row_pass<512>();
    row_pass<1024>();
    row_pass<2048>();
    row_pass<4096>();
    row_pass<8192>();
    column_pass<256>();
    column_pass<512>();
    column_pass<1024>();
    column_pass<2048>();
    std::printf("checked %lld\n", g_checked);
    return 0;
}
