// Host-side check of the split shared-memory slot form of the transforms
// (Slot in device.cuh): wherever a transform pass uses base(lb, g) +
// off(c), the result must equal the padded slot phys(eidx(lb + c, g)).
// Every layout, padding shift (= log2 of the largest radix), transform
// length 2^2..2^14 and tile width with at most 2^15 elements is checked for
// both radix orders.  Prints the number of checked slots; exits non-zero
// on the first mismatch.
#include <cstdio>
#include <cstdlib>
#include <utility>

#include "device.cuh"

using namespace mpa;

static long long g_checked = 0;

static void expect(int got, int want, const char* site, int layout, int L, int G, int psh) {
    ++g_checked;
    if (got != want) {
        std::printf("mismatch at %s: layout %d L %d G %d PSH %d: %d != %d\n", site, layout, L, G, psh, got, want);
        std::exit(1);
    }
}

template <int LAYOUT, int L, int G, int PSH, bool SF, int P, int NP> void passes() {
    if constexpr (P < NP) {
        typedef Sched<L, (1 << PSH)> SC;
        typedef Slot<LAYOUT, L, G, PSH> SL;
        constexpr int R = SC::template radix<SF>(P), NS = SC::template ns<SF>(P);
        if constexpr (P == 0) {  // first-pass scatter j R + r
            for (int j = 0; j < L / R; ++j)
                for (int g = 0; g < G; ++g)
                    for (int r = 0; r < R; ++r)
                        expect(SL::base(j * R, g) + SL::off(r), phys<PSH>(eidx<LAYOUT, L, G>(j * R + r, g)),
                               "scatter", LAYOUT, L, G, PSH);
        } else {
            // reads j + r L/R (middle passes and the last-pass gather)
            if constexpr (SL::template strided<L / R, R>())
                for (int j = 0; j < L / R; ++j)
                    for (int g = 0; g < G; ++g)
                        for (int r = 0; r < R; ++r)
                            expect(SL::base(j, g) + SL::off(r * (L / R)),
                                   phys<PSH>(eidx<LAYOUT, L, G>(j + r * (L / R), g)), "read", LAYOUT, L, G, PSH);
            // middle-pass writes (j - k) R + k + r NS
            if constexpr (P < NP - 1 && SL::template strided<NS, R>())
                for (int j = 0; j < L / R; ++j) {
                    const int k = j & (NS - 1), dst = (j - k) * R + k;
                    for (int g = 0; g < G; ++g)
                        for (int r = 0; r < R; ++r)
                            expect(SL::base(dst, g) + SL::off(r * NS), phys<PSH>(eidx<LAYOUT, L, G>(dst + r * NS, g)),
                                   "write", LAYOUT, L, G, PSH);
                }
        }
        passes<LAYOUT, L, G, PSH, SF, P + 1, NP>();
    }
}

template <int LAYOUT, int PSH, int LOGL, int LOGG> void one() {
    constexpr int L = 1 << LOGL, G = 1 << LOGG;
    if constexpr (L * G <= (1 << 15)) {
        typedef Sched<L, (1 << PSH)> SC;
        if constexpr (SC::NP > 1) {
            passes<LAYOUT, L, G, PSH, true, 0, SC::NP>();
            passes<LAYOUT, L, G, PSH, false, 0, SC::NP>();
        }
    }
}

template <int LAYOUT, int PSH, int LOGL, int... LOGG> void over_g(std::integer_sequence<int, LOGG...>) {
    (one<LAYOUT, PSH, LOGL, LOGG>(), ...);
}
template <int LAYOUT, int PSH, int... LOGL> void over_l(std::integer_sequence<int, LOGL...>) {
    (over_g<LAYOUT, PSH, LOGL + 2>(std::make_integer_sequence<int, 11>{}), ...);
}

int main() {
    over_l<LAYOUT_COL, 5>(std::make_integer_sequence<int, 13>{});
    over_l<LAYOUT_ROW, 5>(std::make_integer_sequence<int, 13>{});
    over_l<LAYOUT_COL, 4>(std::make_integer_sequence<int, 13>{});
    over_l<LAYOUT_ROW, 4>(std::make_integer_sequence<int, 13>{});
    over_l<LAYOUT_COL, 3>(std::make_integer_sequence<int, 13>{});
    over_l<LAYOUT_ROW, 3>(std::make_integer_sequence<int, 13>{});
    std::printf("checked %lld slots\n", g_checked);
    return 0;
}
