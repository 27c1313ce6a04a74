// Host-side check of the packed FP32 convolution form (csrc/taps.h), compiled
// and run by tests/test_tap_pairs.py on the CPU.
//
// The scalar form adds f[k & 1][t] * win[j] into output k of a chunk, with
// t = j - k - off(k & 1), for every window element j and every tap t that
// applies.  The packed form updates outputs 2m and 2m + 1 together from
// window element j with the tap pair tp[j - 2m] (a zero where a tap does not
// apply).  For every filter kind and both chunk widths this checks that the
// pair table gives each output exactly the scalar form's tap for every j,
// that no applying tap lies outside the window, and that each output gets
// every applying tap once.  Prints OK and returns 0 when every check passes.
#include <cstdio>

#include "taps.h"

using namespace wvl;

static int fails = 0;
#define CHECK(c, ...)                           \
    do {                                        \
        if (!(c)) {                             \
            if (fails++ < 10) {                 \
                std::printf("FAIL %s: ", #c);   \
                std::printf(__VA_ARGS__);       \
                std::printf("\n");              \
            }                                   \
        }                                       \
    } while (0)

template <int KIND, int NOUT>
static void check_kind(const char* name) {
    constexpr int NT = KT<KIND>::NT;
    constexpr int W = NOUT + NT - 1 + KT<KIND>::EXTRA;   // window of a chunk
    // distinct, non-zero taps everywhere (also past NT), so a wrong index or
    // a tap that should not apply cannot go unseen
    float f[2][32];
    for (int e = 0; e < 2; ++e)
        for (int t = 0; t < 32; ++t) f[e][t] = 1.0f + 0.5f * e + 0.015625f * t;
    float2 tp[32];
    tap_pairs<KIND>(f, tp);
    int used[NOUT] = {};
    for (int j = -4; j < W + 8; ++j)
        for (int m = 0; m < NOUT / 2; ++m)
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * m + h;
                const int t = j - k - (h ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
                const float want = tap_on<KIND>(t) ? f[h][t] : 0.0f;
                const int d = j - 2 * m;
                float got = 0.0f;
                if (pair_on<KIND>(d)) got = h ? tp[d].y : tp[d].x;
                CHECK(got == want, "%s NOUT %d: j %d output %d tap %d: %g vs %g", name, NOUT, j, k,
                      t, (double)got, (double)want);
                if (want != 0.0f) {
                    CHECK(j >= 0 && j < W, "%s NOUT %d: tap %d of output %d at window element %d",
                          name, NOUT, t, k, j);
                    ++used[k];
                }
            }
    for (int k = 0; k < NOUT; ++k)
        CHECK(used[k] == NT - 2 * KT<KIND>::SKIP, "%s NOUT %d: output %d gets %d taps", name,
              NOUT, k, used[k]);
}

int main() {
    check_kind<K_MF, 8>("magic filter");
    check_kind<K_MF, 16>("magic filter");
    check_kind<K_MFT, 8>("transposed magic filter");
    check_kind<K_MFT, 16>("transposed magic filter");
    check_kind<K_KIN, 8>("kinetic");
    check_kind<K_KIN, 16>("kinetic");
    check_kind<K_SYN, 8>("synthesis");
    check_kind<K_SYN, 16>("synthesis");
    check_kind<K_ANA, 8>("analysis");
    check_kind<K_ANA, 16>("analysis");
    check_kind<K_SYN, 4>("synthesis");
    check_kind<K_KIN, 4>("kinetic");
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
