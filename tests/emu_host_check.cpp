// Host-side checks of the digit arithmetic behind the tensor-core FP64 passes
// (paper_0904_1543_gb300/csrc/emu.cuh), compiled and run by
// tests/test_emu_host.py on the CPU.
//
//  1. quantize + digits: the signed base-1024 digits reconstruct X exactly,
//     stay in range, and X is x on the line's scale to within half a unit.
//  2. build_sched: every filter of the method (the kinetic one at many axis
//     spacings) gets the canonical schedule, and the bounds that make the
//     FP32 partial sums exact hold.
//  3. One window in integer arithmetic as the kernels evaluate it (exact
//     pair sums for diagonals 2..5, FP32 sums for 6..8, 64-bit recombination,
//     the final scaling) against a long-double convolution: the error is
//     within a few units of FP64 rounding of max|f| max|x|.
// Prints OK and returns 0 when every check passes.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "emu.cuh"
#include "wvl.h"

using namespace wvl::emu;

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

// taps of the five kinds as the library sets them (taps f[parity][t])
static void taps(int kind, double hg, const double* h, const double* g, const double* w,
                 const double* a, double f[2][32], int& nt) {
    for (int e = 0; e < 2; ++e)
        for (int t = 0; t < 32; ++t) f[e][t] = 0.0;
    auto H = [&](int j) { return h[j + 7]; };
    auto G = [&](int j) { return g[j + 7]; };
    nt = 16;
    for (int t = 0; t < 16; ++t) {
        if (kind == wvl::K_MF) f[0][t] = f[1][t] = w[15 - t];
        if (kind == wvl::K_MFT) f[0][t] = f[1][t] = w[t];
        if (kind == wvl::K_SYN) {
            f[0][t] = (t % 2 == 0) ? H(8 - t) : G(9 - t);
            f[1][t] = (t % 2 == 0) ? H(7 - t) : G(8 - t);
        }
        if (kind == wvl::K_ANA) {
            f[0][t] = H(t - 7);
            f[1][t] = G(t - 7);
        }
    }
    if (kind == wvl::K_KIN) {
        nt = 29;
        for (int t = 0; t < 29; ++t) f[0][t] = f[1][t] = -a[28 - t] / (2.0 * hg * hg);
    }
}

int main() {
    std::mt19937_64 rng(9041543);
    std::uniform_real_distribution<double> U(-1.0, 1.0);

    // ---------------------------------------------------- 1. digits
    for (int it = 0; it < 1000000; ++it) {
        const double x = U(rng) * std::ldexp(1.0, (int)(rng() % 80) - 40);
        const double big = std::fabs(x) * std::ldexp(1.0, (int)(rng() % 30));
        const int E = scale_of(bexp(big));
        CHECK(std::fabs(x) < std::ldexp(1.0, E), "scale %g %d", x, E);
        const long long X = quantize(x, E);
        CHECK(std::llabs(X) < (1LL << QBITS), "range %lld", X);
        int d[S];
        digits(X, d);
        __int128 R = 0;
        for (int q = 0; q < S; ++q) {
            if (q == 0) CHECK(d[q] >= -512 && d[q] <= 512, "top digit %d", d[q]);
            else CHECK(d[q] >= -512 && d[q] <= 511, "digit %d = %d", q, d[q]);
            R = R * 1024 + d[q];
        }
        CHECK(R == (__int128)X, "reconstruction");
        // |x - X 2^(E - QBITS)| <= half a unit (2^(E - QBITS - 1))
        const long double back = std::ldexp((long double)X, E - QBITS);
        CHECK(std::fabs((long double)x - back) <= std::ldexp(1.0L, E - QBITS - 1), "rounding");
    }
    CHECK(quantize(0.0, 5) == 0, "zero");
    // quantize exactly: the magnitude m 2^(e - 1075 + QBITS - E) rounded half
    // up, in 128-bit integers from the bit pattern (every binade offset from
    // the scale, and the ties)
    {
        std::uniform_int_distribution<int> sh(-6, 70);
        for (int it = 0; it < 2000000; ++it) {
            const int E = (int)(rng() % 200) - 100;
            const int s = sh(rng);                 // x's binade below the scale
            unsigned long long mant = rng() & ((1ULL << 52) - 1);
            if (it % 7 == 0) mant &= ~((1ULL << (rng() % 52)) - 1);   // many trailing zeros: ties
            const double x0 = std::ldexp((double)((1ULL << 52) | mant), E + 1075 - QBITS - s - 1075);
            const double x = (it & 1) ? -x0 : x0;
            if (!(std::fabs(x) < std::ldexp(1.0, E)) || bexp(x) == 0) continue;
            const unsigned long long m = (1ULL << 52) | mant;
            const int r = s;                       // X = m 2^-r
            __int128 ref;
            if (r <= 0) ref = (__int128)m << (-r);
            else if (r >= 100) ref = 0;
            else ref = ((__int128)m + (((__int128)1 << r) >> 1)) >> r;
            const long long got = quantize(x, E);
            CHECK((__int128)(got < 0 ? -got : got) == ref && ((got < 0) == (x < 0) || ref == 0),
                  "quantize exact x %a E %d", x, E);
        }
    }

    // ---------------------------------------------------- 2. schedules
    double h[16], g[16], w[16], a[29];
    int k0 = 0;
    CHECK(wvl_filters(h, g, w, &k0, a) == WVL_OK, "filters");
    std::vector<std::pair<int, double>> cases;
    for (int kind : {wvl::K_MF, wvl::K_MFT, wvl::K_SYN, wvl::K_ANA}) cases.push_back({kind, 0.25});
    for (int i = 0; i < 400; ++i) cases.push_back({wvl::K_KIN, 0.05 + i * 0.005});
    for (auto& c : cases) {
        double f[2][32];
        int nt;
        taps(c.first, c.second, h, g, w, a, f, nt);
        Sched s;
        CHECK(build_sched(f, nt, s), "schedule kind %d h %g", c.first, c.second);
        CHECK(s.npairs == 26 && s.nacc == NACC && s.nexact == NEXACT, "shape %d %d %d", s.npairs,
              s.nacc, s.nexact);
        // pairs in diagonal order, accumulator = diagonal - 2
        for (int i = 0; i < s.npairs; ++i)
            CHECK(s.pacc[i] == s.pp[i] + s.pq[i], "pair %d", i);
    }

    // ---------------------------------------------------- 3. one window
    double worst = 0.0;
    for (int kind : {wvl::K_MF, wvl::K_KIN, wvl::K_SYN}) {
        double f[2][32];
        int nt;
        taps(kind, 0.3, h, g, w, a, f, nt);
        int ebf = 0;
        for (int e = 0; e < 2; ++e)
            for (int t = 0; t < nt; ++t) ebf = std::max(ebf, bexp(f[e][t]));
        const int Ef = scale_of(ebf);
        for (int trial = 0; trial < 2000; ++trial) {
            // one line: values over several decades (a decaying tail)
            std::vector<double> x(nt + 1);
            for (auto& v : x) v = U(rng) * std::pow(10.0, -6.0 * (double)(rng() % 1000) / 1000.0);
            int ebx = 0;
            for (double v : x) ebx = std::max(ebx, bexp(v));
            const int Ex = scale_of(ebx);
            const int e = (int)(rng() & 1);
            long double exact = 0.0L, mag = 0.0L;
            long long D[DMAX + 1] = {0};
            for (int t = 0; t < nt; ++t) {
                const double xv = x[t + (kind == wvl::K_SYN ? e : 0)];
                exact += (long double)f[e][t] * xv;
                mag += std::fabs((long double)f[e][t] * xv);
                int df[S], dx[S];
                digits(quantize(f[e][t], Ef), df);
                digits(quantize(xv, Ex), dx);
                for (int p = 0; p < S; ++p)
                    for (int q = 0; q < S; ++q)
                        if (p + q + 2 <= DMAX) D[p + q + 2] += (long long)df[p] * dx[q];
            }
            // the kernels' recombination
            long long T = 0;
            for (int d = 2; d <= 5; ++d) {
                CHECK(std::llabs(D[d]) < (1LL << 24), "exact diagonal %d = %lld", d, D[d]);
                T += D[d] << (DBITS * (DMAX - d) - TSHIFT);
            }
            float low = 0.f;
            for (int d = 6; d <= DMAX; ++d)
                low = std::fmaf((float)D[d], std::ldexp(1.0f, DBITS * (DMAX - d) - TSHIFT), low);
            T += (long long)std::lrintf(low);
            const long double got = std::ldexp((long double)(double)T, Ex + Ef - OUT_EXP);
            // a few units of FP64 rounding of the line's scale
            const long double scale = std::ldexp(1.0L, Ex + Ef);
            const long double err = std::fabs(got - exact);
            const long double bound = std::ldexp(mag, -52) + 8.0L * std::ldexp(scale, -58);
            CHECK(err <= bound, "window error %Lg > %Lg (kind %d)", err, bound, kind);
            worst = std::max(worst, (double)(err / scale));
        }
    }
    std::printf("worst window error / (max|f| max|x| scale) = %.3g\n", worst);
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("OK\n");
    return 0;
}
