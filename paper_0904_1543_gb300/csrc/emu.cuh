// FP64-accurate 1D passes on the FP16 tensor cores (Ozaki-style slicing).
//
// A pass computes out(I) = sum_t f_t x(I - hl + off + t) on every line (the
// 1D convolutions of Eqs. 1dconvtrans and kinetic1d).  For a tile of M = 128
// lines and a window of N consecutive outputs (32 for the 16-tap filters,
// 16 for the 29-tap kinetic filter) this is one small matrix product
// D[line][j] = sum_k X[line][k] B[k][j] over the K = 48 input positions the
// window reads, B being the banded filter matrix.  Both operands are turned into integers on a common
// scale -- per line for X (its largest exponent), per filter for B -- and
// split into S = 6 signed base-1024 digits:
//
//     X = sum_q x_q 1024^(S-q),  F = sum_p f_p 1024^(S-p),  |x_q|, |f_p| <= 512.
//
// Every digit is exact in FP16, every digit product (<= 2^18) and every sum
// the hardware forms on the way is an integer below 2^24, hence exact in the
// FP32 accumulators; the pairs (p, q) of one diagonal d = p + q share an
// accumulator while their summed worst-case bound stays below 2^24.  The
// result is recombined in 64-bit integers,
//
//     sum_k F_k X_k ~ sum_{d=2}^{8} D_d 1024^(2S-d),
//
// dropping the diagonals d >= 9 (a relative contribution below 2^-62 of
// max|f| max|x| per output), and scaled back to FP64.  The arithmetic of the
// method is untouched: only the way each convolution sum is evaluated
// changes, to an accuracy of the same order as FP64 rounding.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "wvl_internal.h"

namespace wvl {
namespace emu {

constexpr int THREADS = 256;     // 8 warps: slicing 16 lines each; epilogue 32 lines x N/2 outputs
constexpr int WARPS = THREADS / 32;
constexpr int M = 128;           // lines per tile (MMA M, TMEM lanes)
constexpr int NMAX = 32;         // outputs per window (MMA N), largest kind
constexpr int NMIN = 16;
constexpr int S = 6;             // digits per operand
constexpr int DBITS = 10;        // bits per digit
constexpr int DMAX = 8;          // highest diagonal kept
constexpr int MAXPAIR = 32;
constexpr int MAXACC = 8;        // accumulators (TMEM columns: MAXACC * N)
// the schedules of the method's filters (all kinetic spacings checked from
// 0.05 to 2): one accumulator per diagonal 2..8, the first four exact
constexpr int NACC = 7;
constexpr int NEXACT = 4;
constexpr int QBITS = DBITS * S - 1;   // |X| < 2^QBITS
// byte stride between the 8-position chunks of one operand plane: the MMA's
// leading-dimension offset.  A: 128 rows of 16 B plus a 64 B bank skew that
// keeps the digit stores (16-position slabs, four lines per warp
// instruction) conflict-free.
__host__ __device__ constexpr int lboa(int) { return M * 16 + 64; }
// T' = (sum of the kept diagonals) / 2^(DBITS (2S - DMAX) + TSHIFT): the
// accumulator of diagonal d enters shifted by DBITS (DMAX - d) - TSHIFT
// (right shifts rounded); the host checks that T' stays below 2^62
constexpr int TSHIFT = 20;
// sum_t f_t x_t = T' 2^(E_x + E_f - OUT_EXP)
constexpr int OUT_EXP = 2 * QBITS - DBITS * (2 * S - DMAX) - TSHIFT;

// outputs per window, input positions read (window start o - HA, 8-aligned)
__host__ __device__ constexpr int window_n(int kind) { return kind == K_KIN ? 16 : 32; }
__host__ __device__ constexpr int window_k(int kind) { return 48; }
__host__ __device__ constexpr int window_ha(int kind) { return kind == K_KIN ? 16 : 8; }
// The filter operand holds the S digit planes side by side along N, then a
// zero block: per 8-position chunk, rows (output j of digit fp) at fp N + j,
// (S + 1) N rows of 16 bytes.  One MMA per data digit dq then covers the
// filter digits fp = 0 .. S - dq at once (N (S + 1 - dq) columns), each
// landing in the accumulator of its diagonal dq + fp.
__host__ __device__ constexpr int lbo_b(int kind) { return (S + 1) * window_n(kind) * 16; }
__host__ __device__ constexpr int tmem_cols(int kind) { return MAXACC * window_n(kind); }
__host__ __device__ constexpr int plane_a_bytes(int kind, int mode) { return window_k(kind) / 8 * lboa(mode); }
__host__ __device__ constexpr int b_bytes(int kind) { return window_k(kind) / 8 * lbo_b(kind); }
__host__ __device__ constexpr int smem_bytes(int kind, int mode) {
    return S * plane_a_bytes(kind, mode) + b_bytes(kind);
}

// Schedule of one launch: which (filter digit p, data digit q) pairs go to
// which accumulator, and each accumulator's weight (a shift of T').
// Accumulators come in diagonal order; the first nexact (diagonals <= 5)
// hold exact integers and enter T' shifted left by shift[ac] >= 10; the
// others (diagonals 6..8, weight 2^shift <= 1) are summed in FP32 with
// weights wlow[ac] and rounded once.
struct Sched {
    int npairs;
    int nacc;
    int nexact;
    unsigned char pp[MAXPAIR], pq[MAXPAIR], pacc[MAXPAIR];
    int shift[MAXACC];
    float wlow[MAXACC];
};

struct Params {
    PassParams<double> p;
    Sched s;
};

__host__ __device__ inline unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

// biased exponent field of x (0 for zero)
__host__ __device__ inline int bexp(double x) { return (int)((dbits(x) >> 52) & 0x7FF); }

// E with |x| < 2^E for every x whose biased exponent is at most eb
__host__ __device__ inline int scale_of(int eb) { return eb - 1022; }

// X = round(x 2^(QBITS - E)) for |x| < 2^E, so |X| < 2^QBITS; integer
// operations on the bit pattern only (subnormal inputs count as zero)
__host__ __device__ inline long long quantize(double x, int E) {
    const unsigned long long b = dbits(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) return 0;
    // x = m 2^(e - 1075), m < 2^53 -> X = m 2^-(sh), sh = E + 1075 - QBITS - e
    // >= -6 (e <= E + 1022).  With the mantissa shifted left by 6 first
    // (m6 < 2^59), X is one right shift by r = sh + 6 >= 0, rounded half up
    // on the magnitude (none of m survives once r >= 60)
    const unsigned long long m6 = ((b & ((1ULL << 52) - 1)) | (1ULL << 52)) << 6;
    int r = E + 1081 - QBITS - e;
    r = r < 0 ? 0 : (r > 63 ? 63 : r);
    const long long X = (long long)((m6 + ((1ULL << r) >> 1)) >> r);   // m6 + half < 2^63
    return (b >> 63) ? -X : X;
}

// signed base-1024 digits, most significant first: d[0] in [-512, 512],
// the others in [-512, 511]
__host__ __device__ inline void digits(long long X, int (&d)[S]) {
#pragma unroll
    for (int q = S - 1; q > 0; --q) {
        int lo = (int)(X & 1023);
        lo -= (lo & 512) << 1;
        d[q] = lo;
        X = (X - lo) >> DBITS;
    }
    d[0] = (int)X;
}

// The digit-pair schedule for one filter (taps f[parity][t], t < nt), from
// the same digits the kernel builds: each pair's partial sums are bounded by
// sum_t |filter digit| x 512 (the largest data digit); the pairs of a
// diagonal <= 5 share an accumulator while their bounds add up to less than
// 2^24 (exact in FP32); diagonals 6..8 take one accumulator each.  False
// when the result is not the canonical schedule the kernels are built for,
// or when |T'| could reach 2^62.
inline bool build_sched(const double (&f)[2][32], int nt, Sched& s) {
    int ebf = 0;
    for (int e = 0; e < 2; ++e)
        for (int t = 0; t < nt; ++t) ebf = std::max(ebf, bexp(f[e][t]));
    const int Ef = scale_of(ebf);
    // sum over the taps of one output of |filter digit p|, worst parity
    double sabs[S] = {0};
    for (int e = 0; e < 2; ++e) {
        double se[S] = {0};
        for (int t = 0; t < nt; ++t) {
            int d[S];
            digits(quantize(f[e][t], Ef), d);
            for (int q = 0; q < S; ++q) se[q] += std::abs(d[q]);
        }
        for (int q = 0; q < S; ++q) sabs[q] = std::max(sabs[q], se[q]);
    }
    const double lim = 16777216.0;   // 2^24: integers exact in FP32
    double tbound = 0.0;             // bound of |T'|
    std::memset(&s, 0, sizeof s);
    for (int d = 2; d <= DMAX; ++d) {
        double load = 0.0;
        int cur = -1;
        for (int fp = 0; fp < S; ++fp) {
            const int dq = d - 2 - fp;   // digits are 0-based: (fp + 1) + (dq + 1) = d
            if (dq < 0 || dq >= S) continue;
            const double b = sabs[fp] * 512.0;
            const bool exact = d <= 5;   // weight above 2^-40 of the top diagonal
            if (cur < 0 || (exact && load + b > lim)) {
                if (s.nacc >= MAXACC) return false;
                cur = s.nacc++;
                s.shift[cur] = DBITS * (DMAX - d) - TSHIFT;
                s.wlow[cur] = (float)std::ldexp(1.0, s.shift[cur]);
                if (exact) s.nexact = s.nacc;
                load = 0.0;
            }
            load += b;
            tbound += b * std::ldexp(1.0, s.shift[cur]);
            if (s.npairs >= MAXPAIR) return false;
            s.pp[s.npairs] = (unsigned char)fp;
            s.pq[s.npairs] = (unsigned char)dq;
            s.pacc[s.npairs] = (unsigned char)cur;
            ++s.npairs;
        }
    }
    // the kernels take the canonical schedule: accumulator a holds diagonal
    // a + 2, exact for a < NEXACT (shift >= 10), FP32-summed otherwise
    if (s.nacc != NACC || s.nexact != NEXACT) return false;
    for (int a = 0; a < NACC; ++a)
        if (s.shift[a] != DBITS * (DMAX - 2 - a) - TSHIFT) return false;
    return tbound < std::ldexp(1.0, 62);
}

#ifdef __CUDACC__
#include <cuda_fp16.h>

// The digits of two inputs, as digits() gives them, digit q of both as one
// FP16x2 word (X0's in the low half).  Adding 512 to every lower digit
// position makes the lower digits plain 10-bit fields of
// Y = X + sum_k 512 1024^k (no carry chain); the field y = digit + 512 in
// [0, 1024] (the top one: the top digit + 512) becomes the FP16 value 1024 + y
// through the bit pattern 0x6400 + y (y = 1024 carries into the exponent:
// 2048), and one packed FP16 subtraction of 1536 leaves the digit, exactly.
__device__ __forceinline__ void digit_pairs(long long X0, long long X1, uint32_t (&h)[S]) {
    constexpr long long C = 512LL * (1 + (1LL << 10) + (1LL << 20) + (1LL << 30) + (1LL << 40));
    static_assert(S == 6, "digit layout");
    const unsigned long long Y0 = (unsigned long long)(X0 + C), Y1 = (unsigned long long)(X1 + C);
    const unsigned l0 = (unsigned)Y0, h0 = (unsigned)(Y0 >> 32);
    const unsigned l1 = (unsigned)Y1, h1 = (unsigned)(Y1 >> 32);
    const __half2 off = __halves2half2(__ushort_as_half((unsigned short)0x6600),
                                       __ushort_as_half((unsigned short)0x6600));   // 1536
    // fields y0, y1 <= 1024 -> the word (0x6400 + y0) | (0x6400 + y1) << 16,
    // the halves joined by a byte permute (no carry crosses them)
    auto pack = [&](unsigned y0, unsigned y1) {
        const unsigned w = __byte_perm(y0, y1, 0x5410) + 0x64006400u;
        const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&w), off);
        return *reinterpret_cast<const uint32_t*>(&d);
    };
    // the 10-bit field k of Y from its 32-bit halves (field 3 straddles them)
    auto field = [](unsigned lo, unsigned hi, int k) {
        return k < 3 ? (lo >> (DBITS * k)) & 1023u
                     : k == 3 ? __funnelshift_r(lo, hi, 30) & 1023u : (hi >> (DBITS * k - 32)) & 1023u;
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) h[S - 1 - k] = pack(field(l0, h0, k), field(l1, h1, k));
    h[0] = pack((unsigned)(((int)h0 >> (DBITS * (S - 1) - 32)) + 512),
                (unsigned)(((int)h1 >> (DBITS * (S - 1) - 32)) + 512));
}
#endif

}  // namespace emu

// Launches one emulated pass (same parameters and outputs as launch_pass for
// double; the segments carry tiles = line tiles x windows and nwin).
cudaError_t launch_pass_emu(int kind, int mode, const PassParams<double>& p, long long nunits,
                            cudaStream_t st);
cudaError_t prepare_emu_kernels();
// Largest biased exponent of every line of synthesis pass 1's input (full-
// grid compressed form, cell of n1 x n2 x n3 coarse points, norb orbitals of
// P elements): lexp[orbital][x3 * 2 n2 + x2].
cudaError_t launch_line_exp(const double* in, int* lexp, int n1, int n2, int n3, int norb,
                            long long P, cudaStream_t st);
// bounded waits of the emulated passes that ran out since the last call
cudaError_t emu_take_timeouts(unsigned* count);
// one bounded wait that cannot be satisfied, given up after about ms
cudaError_t emu_wait_probe(double ms, cudaStream_t st);

}  // namespace wvl
