// The 1D "convolve + transpose" pass (Eqs. 1dconvtrans, kinetic1d) for
// sm_103a, templated on the element type, the operator, the epilogue and the
// number of consecutive outputs per thread.
//
// A job is a tile of LT consecutive lines of one orbital.  The CTA keeps the
// whole periodic lines in shared memory, extended by the left/right halos,
// which are copied from their wrapped positions -- this is how the periodic
// boundary is applied.  A thread computes R consecutive outputs of one line
// from a register window of R + NT - 1 (+1 for the two-phase wavelet filters)
// shared-memory values; taps are kernel parameters (constant bank) and the
// tap indices are compile-time, so the inner loop is loads and FMAs only.
// Outputs go to F[I][a] with the line index fastest, so each warp's stores
// are coalesced (LT contiguous elements).
//
// The kernel is persistent and double-buffered: while it computes job k from
// one staging buffer, the asynchronous copies (cp.async) of job k+1 fill the
// other, so the arithmetic pipe does not wait for a staging phase.
#pragma once
#include <cuda_runtime.h>

#include "taps.h"
#include "wvl_internal.h"

namespace wvl {

constexpr int NWARPS = NTHREADS / 32;

// Row slot of input position 0: the left halo, rounded up to a 16-byte
// boundary for FP32 so that the line's interior is staged with 16-byte
// copies; the window of a chunk then starts D = row_hl - HL words later.
template <typename T, int KIND>
__host__ __device__ constexpr int row_hl() {
    return sizeof(T) == 4 ? (KT<KIND>::HL + 3) / 4 * 4 : KT<KIND>::HL;
}

// Reductions.  Energies (sums over the grid) accumulate in FP64 in both
// forms: in the FP32 form every term is an FP32 chain of at most 32 products
// of the convolution outputs, converted exactly and added to a double.  The
// FP32 form's density (a sum over orbitals at every point) is carried per
// thread in a compensated FP32 pair (Knuth two-sum, about 48 significant
// bits) and in FP64 from the flush on: one FP64 addition per orbital and
// point instead measured 14.7 % slower on the fused chain, with the same
// density error (the FP32 convolutions dominate it).
struct FF { float hi, lo; };
__device__ __forceinline__ void ff_add(FF& a, float x) {
    float s = a.hi + x;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (x - bb);
    a.hi = s;
    a.lo += e;
}

// two compensated pairs at once with packed FP32 arithmetic (two adds per
// lane per instruction): the same two-sum, s - a computed as s + (-1) a
struct FF2 { float2 hi{0.f, 0.f}, lo{0.f, 0.f}; };
__device__ __forceinline__ void ff2_add(FF2& a, float2 x) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 s = __fadd2_rn(a.hi, x);
    const float2 bb = __ffma2_rn(a.hi, m1, s);     // s - hi
    const float2 t = __ffma2_rn(bb, m1, s);        // s - bb
    const float2 e1 = __ffma2_rn(t, m1, a.hi);     // hi - (s - bb)
    const float2 e2 = __ffma2_rn(bb, m1, x);       // x - bb
    a.lo = __fadd2_rn(a.lo, __fadd2_rn(e1, e2));
    a.hi = s;
}
__device__ __forceinline__ double ff2_get(const FF2& a, int c) {
    return c ? (double)a.hi.y + (double)a.lo.y : (double)a.hi.x + (double)a.lo.x;
}

// energy accumulator: FP64 in both forms
template <typename T> struct Acc;
template <> struct Acc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void fma_add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double get() const { return v; }
    __device__ __forceinline__ void reset() { v = 0.0; }
};
template <> struct Acc<float> {
    double v = 0.0;
    __device__ __forceinline__ void add(float x) { v += (double)x; }
    __device__ __forceinline__ void add(double x) { v += x; }
    // a scalar-product term: the FP32 x FP32 product, exact in FP64
    __device__ __forceinline__ void fma_add(float a, float b) { v = fma((double)a, (double)b, v); }
    __device__ __forceinline__ double get() const { return v; }
    __device__ __forceinline__ void reset() { v = 0.0; }
};

// density accumulator: FP64, or a compensated FP32 pair in the FP32 form;
// add() takes occ psi^2 formed in the form's precision
template <typename T> struct RhoAcc;
template <> struct RhoAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double get() const { return v; }
    __device__ __forceinline__ void reset() { v = 0.0; }
};
template <> struct RhoAcc<float> {
    FF f{0.f, 0.f};
    __device__ __forceinline__ void add(float x) { ff_add(f, x); }
    __device__ __forceinline__ double get() const { return (double)f.hi + (double)f.lo; }
    __device__ __forceinline__ void reset() { f.hi = 0.f; f.lo = 0.f; }
};

__device__ __forceinline__ double block_sum(double v, double* red) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        #pragma unroll
        for (int w = 0; w < NWARPS; ++w) t += red[w];
    }
    __syncthreads();
    return t;
}

// ------------------------------------------------------ asynchronous copies
template <typename T>
__device__ __forceinline__ void cp_async(T* smem_dst, const T* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// copy, or zero-fill the destination when the source does not exist
template <typename T>
__device__ __forceinline__ void cp_async_or_zero(T* smem_dst, const T* gsrc, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const unsigned nbytes = valid ? (unsigned)sizeof(T) : 0u;
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc),
                     "r"(nbytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc),
                     "r"(nbytes) : "memory");
}
// 16 or 8 bytes, both addresses aligned to the size
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// R consecutive elements of one line from global memory; 16-byte loads when
// all R exist and the line start is 16-byte aligned (vec)
template <typename T, int R>
__device__ __forceinline__ void load_run(const T* __restrict__ src, int i, int n, bool vec,
                                         T (&v)[R]) {
    if (vec && i + R <= n) {
        constexpr int PER = 16 / (int)sizeof(T);
        #pragma unroll
        for (int q = 0; q < R / PER; ++q) {
            if constexpr (sizeof(T) == 4) {
                const float4 f = reinterpret_cast<const float4*>(src + i)[q];
                v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
            } else {
                const double2 d = reinterpret_cast<const double2*>(src + i)[q];
                v[2 * q] = d.x; v[2 * q + 1] = d.y;
            }
        }
        return;
    }
    #pragma unroll
    for (int r = 0; r < R; ++r)
        if (i + r < n) v[r] = src[i + r];
}

// R outputs of one line from the shared-memory row (srow[j] <-> position
// i0 - HL + j); acc must hold the initial values.
template <typename T, int KIND, int R>
__device__ __forceinline__ void conv_chunk(const T* __restrict__ srow,
                                           const PassParams<T>& p, T (&acc)[R]) {
    constexpr int NT = KT<KIND>::NT;
    constexpr int W = R + NT - 1 + KT<KIND>::EXTRA;
    if constexpr (sizeof(T) == 4) {
        // FP32: the window in 16-byte loads from the chunk's aligned start
        // (rows and chunks are 16-byte aligned, and the row stride keeps the
        // 8 lanes of a phase on distinct banks); the taps begin D words in
        constexpr int D = row_hl<T, KIND>() - KT<KIND>::HL;
        constexpr int W4 = (W + D + 3) / 4 * 4;
        float win[W4];
        #pragma unroll
        for (int q = 0; q < W4 / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(srow)[q];
            win[4 * q] = v.x;
            win[4 * q + 1] = v.y;
            win[4 * q + 2] = v.z;
            win[4 * q + 3] = v.w;
        }
        // outputs 2m, 2m + 1: one packed FMA per window element
        static_assert(R % 2 == 0, "output pairs");
        float2 a2[R / 2];
        #pragma unroll
        for (int m = 0; m < R / 2; ++m) a2[m] = make_float2(acc[2 * m], acc[2 * m + 1]);
        #pragma unroll
        for (int j = 0; j < W; ++j) {
            const float2 ww = make_float2(win[j + D], win[j + D]);
            #pragma unroll
            for (int m = 0; m < R / 2; ++m)
                if (pair_on<KIND>(j - 2 * m)) a2[m] = __ffma2_rn(p.tp[j - 2 * m], ww, a2[m]);
        }
        #pragma unroll
        for (int m = 0; m < R / 2; ++m) {
            acc[2 * m] = a2[m].x;
            acc[2 * m + 1] = a2[m].y;
        }
        return;
    }
    #pragma unroll
    for (int j = 0; j < W; ++j) {
        const T v = srow[j];
        #pragma unroll
        for (int r = 0; r < R; ++r) {
            const int t = j - r - ((r & 1) ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
            if (t >= KT<KIND>::SKIP && t < NT - KT<KIND>::SKIP) acc[r] = fma(p.f[r & 1][t], v, acc[r]);
        }
    }
}

// Position of coarse point (i1, i2, i3) in the stored compressed vector:
// the scaling coefficient c^0 sits at k, c^mu (mu >= 1) at ncoarse + 7 k + mu - 1;
// -1 if the point is outside the localisation region or the box of free /
// surface boundary conditions (whose cell is padded by bo_d points per side
// along each free axis d).
template <typename T>
__device__ __forceinline__ int stored_index(const Seg<T>& S, long long ci, int i1, int i2,
                                            int i3, int mu) {
    if (S.bx1 > 0) {
        const int j1 = i1 - S.bo1, j2 = i2 - S.bo2, j3 = i3 - S.bo3;
        if ((unsigned)j1 >= (unsigned)S.bx1 || (unsigned)j2 >= (unsigned)S.bx2 ||
            (unsigned)j3 >= (unsigned)S.bx3)
            return -1;
        return (j3 * S.bx2 + j2) * S.bx1 + j1;
    }
    return (mu == 0) ? S.mapc[ci] : S.mapf[ci];
}

// Linear coarse index, in the compressed layout's cell, of coarse point
// (j1, j2, j3) of the arrays a pass works on: the same point, or with free
// lines over a region's box, the box point shifted by the box origin and
// wrapped into the periodic cell.
template <typename T>
__device__ __forceinline__ long long cell_ci(const Seg<T>& S, int j1, int j2, int j3) {
    if (S.gc1 == 0) return ((long long)j3 * S.n2 + j2) * S.n1 + j1;
    int g1 = j1 + S.go1, g2 = j2 + S.go2, g3 = j3 + S.go3;
    if (g1 >= S.gc1) g1 -= S.gc1;
    if (g2 >= S.gc2) g2 -= S.gc2;
    if (g3 >= S.gc3) g3 -= S.gc3;
    return ((long long)g3 * S.gc2 + g2) * S.gc1 + g1;
}

// ------------------------------------------------------------------- jobs
struct Job {
    long long unit;   // global work unit
    int si;           // segment
    int tile;
    int orb;          // orbital within the segment
    int oe;           // one past the last orbital of the unit
    bool valid;
};

template <typename T, int MODE>
__device__ __forceinline__ Job make_job(const PassParams<T>& p, long long u) {
    Job J;
    J.unit = u;
    J.valid = u < p.nunits;
    if (!J.valid) return J;
    int si = 0;
    #pragma unroll 1
    while (si + 1 < p.nseg && u >= p.seg[si + 1].blk0) ++si;
    const Seg<T>& S = p.seg[si];
    const long long loc = u - S.blk0;
    J.si = si;
    J.tile = (int)(loc % S.tiles);
    const int grp = (int)(loc / S.tiles);
    if (MODE == M_POT) {
        J.orb = grp * S.opg;
        J.oe = min(S.norb, J.orb + S.opg);
    } else {
        J.orb = grp;
        J.oe = grp + 1;
    }
    return J;
}

template <typename T, int MODE>
__device__ __forceinline__ Job next_job(const PassParams<T>& p, const Job& J) {
    if (J.orb + 1 < J.oe) {
        Job K = J;
        K.orb += 1;
        return K;
    }
    return make_job<T, MODE>(p, J.unit + gridDim.x);
}

// Issue the copies of job J's lines (and wrapped halos) into buf.
template <typename T, int KIND, int MODE>
__device__ __forceinline__ void stage(const PassParams<T>& p, const Job& J, T* buf) {
    const Seg<T>& S = p.seg[J.si];
    constexpr int hl = row_hl<T, KIND>();
    const int n = S.n, rowlen = S.rowlen, LT = p.LT;
    const int a0 = J.tile * LT;
    const int lt = min(LT, S.N - a0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long P = S.P;
    #pragma unroll 1
    for (int r = warp; r < LT; r += NWARPS) {
        T* row = buf + r * rowlen;
        if (r >= lt) {
            for (int j = lane; j < rowlen; j += 32) row[j] = T(0);
            continue;
        }
        const int a = a0 + r;
        if (S.nin > 0) {
            // free lines: row slot j holds input element j - hl + inoff of a
            // line of nin, zero outside it (no wrap)
            const int nin = S.nin;
            if (MODE == M_UNCOMP) {
                // the box's interleaved coarse array, line a = (x3, x2) of it
                const int x3 = a / S.N2, x2 = a - x3 * S.N2;
                const int mu23 = 2 * (x2 & 1) + 4 * (x3 & 1);
                const T* cc = S.in + (long long)J.orb * S.clen;
                const T* cf = cc + S.ncoarse;
                const long long cb = ((long long)(x3 >> 1) * S.n2 + (x2 >> 1)) * S.n1;
                #pragma unroll 1
                for (int j = lane; j < rowlen; j += 32) {
                    const int x = j - hl + S.inoff;
                    bool ok = (unsigned)x < (unsigned)nin;
                    const int mu = mu23 + (x & 1);
                    long long k = cb + (x >> 1);
                    if (ok && S.mapc != nullptr) {
                        // region: the point's position in the stored vector, -1 off it
                        k = stored_index(S, cell_ci(S, x >> 1, x2 >> 1, x3 >> 1), 0, 0, 0, mu);
                        ok = k >= 0;
                    }
                    const T* src = !ok ? cc : ((mu == 0) ? cc + k : cf + k * 7 + mu - 1);
                    cp_async_or_zero(row + j, src, ok);
                }
            } else {
                const T* src = S.in + (long long)J.orb * S.Pin + (long long)a * nin;
                #pragma unroll 1
                for (int j = lane; j < rowlen; j += 32) {
                    const int x = j - hl + S.inoff;
                    const bool ok = (unsigned)x < (unsigned)nin;
                    cp_async_or_zero(row + j, ok ? src + x : src, ok);
                }
            }
            continue;
        }
        // source position of row slot j is x = (j - hl) mod n
        int x = lane - hl;
        while (x < 0) x += n;
        while (x >= n) x -= n;
        if (MODE == M_UNCOMP) {
            // line a = (x3, x2) of the interleaved coarse array; element x1 of
            // it is c^mu[i3][i2][i1], mu = a1 + 2 a2 + 4 a3
            const int x3 = a / S.N2, x2 = a - x3 * S.N2;
            const int mu23 = 2 * (x2 & 1) + 4 * (x3 & 1);
            const T* cc = S.in + (long long)J.orb * S.clen;
            const T* cf = cc + S.ncoarse;
            const long long cb = ((long long)(x3 >> 1) * S.n2 + (x2 >> 1)) * S.n1;
            if (S.mapc == nullptr && S.bx1 == 0) {
                #pragma unroll 1
                for (int j = lane; j < rowlen; j += 32) {
                    const int mu = mu23 + (x & 1);
                    const long long ci = cb + (x >> 1);
                    cp_async(row + j, (mu == 0) ? cc + ci : cf + ci * 7 + mu - 1);
                    x += 32;
                    while (x >= n) x -= n;
                }
            } else {
                // region or box: coefficients off it are zero
                #pragma unroll 1
                for (int j = lane; j < rowlen; j += 32) {
                    const int mu = mu23 + (x & 1);
                    const long long ci = S.gc1 ? cell_ci(S, x >> 1, x2 >> 1, x3 >> 1) : cb + (x >> 1);
                    const int k = stored_index(S, ci, x >> 1, x2 >> 1, x3 >> 1, mu);
                    const T* src = (k < 0) ? cc : ((mu == 0) ? cc + k : cf + (long long)k * 7 + mu - 1);
                    cp_async_or_zero(row + j, src, k >= 0);
                    x += 32;
                    while (x >= n) x -= n;
                }
            }
        } else if (sizeof(T) == 4) {
            // FP32: groups of four row slots; 16-byte copies where the source
            // is 16-byte aligned and does not wrap, 8-byte where it is even
            const T* src = S.in + (long long)J.orb * P + (long long)a * n;
            const bool lines4 = (n & 3) == 0;   // every line starts 16-byte aligned
            int x4 = (4 * lane - hl) % n;         // source of row slot j, kept in [0, n)
            if (x4 < 0) x4 += n;
            #pragma unroll 1
            for (int j = 4 * lane; j < rowlen; j += 128, x4 += 128) {
                while (x4 >= n) x4 -= n;
                if (lines4 && (x4 & 3) == 0 && x4 + 3 < n && j + 3 < rowlen) {
                    cp_async16(row + j, src + x4);
                } else if ((n & 1) == 0 && (x4 & 1) == 0 && x4 + 3 < n && j + 3 < rowlen) {
                    cp_async8(row + j, src + x4);
                    cp_async8(row + j + 2, src + x4 + 2);
                } else {
                    #pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (j + e >= rowlen) break;
                        int xe = x4 + e;
                        while (xe >= n) xe -= n;
                        cp_async(row + j + e, src + xe);
                    }
                }
            }
        } else {
            const T* src = S.in + (long long)J.orb * P + (long long)a * n;
            #pragma unroll 1
            for (int j = lane; j < rowlen; j += 32) {
                cp_async(row + j, src + x);
                x += 32;
                while (x >= n) x -= n;
            }
        }
    }
}

template <typename T, int KIND, int MODE, int R>
__global__ void __launch_bounds__(NTHREADS)
pass_kernel(const __grid_constant__ PassParams<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const bufs = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[NWARPS];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int LT = p.LT;
    constexpr int hl = row_hl<T, KIND>();   // row slot of input position 0
    const int spw = 32 / LT;
    const int line = lane & (LT - 1);
    const int slot = warp * spw + lane / LT;
    const int nslots = NWARPS * spw;
    constexpr bool KM = (MODE == M_KMID || MODE == M_KLAST);
    // FP32 potential pass: the density sums (compensated pairs) live in
    // shared memory after the two staging buffers, slot [I][line] owned by
    // the thread computing output I of that line, which keeps the kernel's
    // registers (and so its occupancy) at the level of the plain passes; the
    // FP64 pass keeps them in registers
    constexpr bool RSM = (MODE == M_POT) && sizeof(T) == 4;
    constexpr int CPT = (MODE == M_POT && !RSM) ? pot_out<T>() / R : 1;
    float2* const rsm = reinterpret_cast<float2*>(smem_raw + 2 * (size_t)p.bufelems * sizeof(T));

    Job cur = make_job<T, MODE>(p, blockIdx.x);
    if (!cur.valid) return;
    stage<T, KIND, MODE>(p, cur, bufs);
    cp_commit();

    RhoAcc<T> racc[RSM ? 1 : CPT][RSM ? 1 : R];   // M_POT (FP64): density per owned output
    int b = 0;

    #pragma unroll 1
    while (true) {
        const Job nxt = next_job<T, MODE>(p, cur);
        if (nxt.valid) {
            stage<T, KIND, MODE>(p, nxt, bufs + (b ^ 1) * p.bufelems);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();

        // ---------------------------------------------- compute job cur
        const Seg<T>& S = p.seg[cur.si];
        const int n = S.n, N = S.N, rowlen = S.rowlen;
        const int a0 = cur.tile * LT;
        const int lt = min(LT, N - a0);
        const bool line_ok = line < lt;
        const int nchunks = (n + R - 1) / R;
        const long long P = S.P;
        const int orb = cur.orb;
        const long long obase = (long long)orb * P;
        const T* srow_line = bufs + b * p.bufelems + line * rowlen;
        Acc<T> e;   // energy partial of this orbital
        double occ = 0.0;
        if (MODE == M_POT) occ = S.occ ? S.occ[orb] : 1.0;
        // M_COMP for the adjoint of E_loc: H psi scaled by 2 occ g
        T osc = T(1);
        if (MODE == M_COMP && S.gscale != nullptr) osc = T(2.0 * S.occ[orb] * S.gscale[0]);
        // FP32 potential pass: the first orbital of the unit starts the sums
        const bool first_orb = RSM && orb == (int)((cur.unit - S.blk0) / S.tiles) * S.opg;
        // index of output I of this line in V and rho: (I + vo3) vplane + vline,
        // the output's own index I N + a unless V and rho live on another grid
        // (free lines)
        long long vline = a0 + line, vplane = N;
        int vo3 = 0, vn3 = 0x7fffffff;
        if (MODE == M_POT && S.vN1 > 0) {
            const int aa = a0 + line, X2 = aa / S.N1, X1 = aa - X2 * S.N1;
            int w1 = X1 + S.vo1, w2 = X2 + S.vo2;
            if (w1 >= S.vN1) w1 -= S.vN1;
            if (w2 >= S.vN2) w2 -= S.vN2;
            vline = (long long)w2 * S.vN1 + w1;
            vplane = (long long)S.vN1 * S.vN2;
            vo3 = S.vo3;
            vn3 = S.vN3;
        }
        auto vidx = [&](int I) -> long long {
            int z = I + vo3;
            if (z >= vn3) z -= vn3;
            return (long long)z * vplane + vline;
        };

        // K_{p-1} of the thread's next chunk, fetched one chunk ahead
        T kv[R];
        #pragma unroll
        for (int r = 0; r < R; ++r) kv[r] = T(0);
        const T* kline = nullptr;
        // line starts 16-byte aligned: the orbital stride P is a multiple of 8
        const bool kvec = (n % (16 / (int)sizeof(T))) == 0;
        if (KM && S.in2 != nullptr && line_ok) {
            kline = S.in2 + obase + (long long)(a0 + line) * n;
            load_run<T, R>(kline, slot * R, n, kvec, kv);
        }

        // M_POT: CPT * nslots >= nchunks (launcher guarantees), so the outer
        // loop runs once and racc[cc] always maps to the same outputs.
        #pragma unroll 1
        for (int cbase = slot; cbase < nchunks; cbase += nslots * CPT) {
            #pragma unroll
            for (int cc = 0; cc < CPT; ++cc) {
                const int c = cbase + cc * nslots;
                if (c >= nchunks) continue;
                const int i0 = c * R;
                T acc[R];
                #pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = KM ? kv[r] : T(0);
                if (MODE == M_KMID && S.in2 == nullptr && S.eps != nullptr) {
                    // K_0 = -eps s: the Helmholtz operator of the preconditioner
                    const T me = T(-S.eps[orb]);
                    #pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] = me * srow_line[hl + i0 + r];
                }
                if (KM && kline != nullptr) load_run<T, R>(kline, (c + nslots) * R, n, kvec, kv);
                conv_chunk<T, KIND, R>(srow_line + i0, p, acc);
                if (!line_ok) continue;
                if (MODE == M_COMP && S.gscale != nullptr) {
                    // the adjoint of E_loc: H psi scaled by 2 occ g (a uniform branch,
                    // so the plain analysis pass pays nothing for it)
                    #pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] *= osc;
                }
                if (MODE == M_PLAIN || MODE == M_UNCOMP) {
                    // transposed store: output I of this line at I * N
                    T* op = S.out + obase + (long long)i0 * N + a0 + line;
                    if (i0 + R <= n) {
                        #pragma unroll
                        for (int r = 0; r < R; ++r) op[(long long)r * N] = acc[r];
                    } else {
                        #pragma unroll
                        for (int r = 0; r < R; ++r)
                            if (i0 + r < n) op[(long long)r * N] = acc[r];
                    }
                    continue;
                }
                const long long oidx0 = (long long)i0 * N + a0 + line;
                T ech = T(0);   // the chunk's energy terms, then added in FP64
                #pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int I = i0 + r;
                    if (I >= n) continue;
                    const long long oidx = oidx0 + (long long)r * N;
                    if (MODE == M_PLAIN || MODE == M_UNCOMP) {
                        S.out[obase + oidx] = acc[r];
                    } else if (MODE == M_COMP) {
                        // output (X3 = I, a = X2 * N1 + X1) -> compressed position
                        const int a = a0 + line;
                        const int X2 = a / S.N1, X1 = a - X2 * S.N1;
                        const int mu = (X1 & 1) + 2 * (X2 & 1) + 4 * (I & 1);
                        const long long ci =
                            ((long long)(I >> 1) * S.n2 + (X2 >> 1)) * S.n1 + (X1 >> 1);
                        T* cc0 = S.out + (long long)orb * S.clen;
                        const T val = acc[r];
                        if (S.mapc == nullptr && S.bx1 == 0) {
                            if (mu == 0) cc0[ci] = val;
                            else cc0[S.ncoarse + ci * 7 + mu - 1] = val;
                        } else {
                            // region or box: only the stored coefficients
                            const long long cg = S.gc1 ? cell_ci(S, X1 >> 1, X2 >> 1, I >> 1) : ci;
                            const int k = stored_index(S, cg, X1 >> 1, X2 >> 1, I >> 1, mu);
                            if (k >= 0) {
                                if (mu == 0) cc0[k] = val;
                                else cc0[S.ncoarse + (long long)k * 7 + mu - 1] = val;
                            }
                        }
                    } else if (MODE == M_KMID) {
                        S.out[obase + oidx] = acc[r];
                        S.out2[obase + oidx] = srow_line[hl + I];
                    } else if (MODE == M_KLAST) {
                        if (S.out) S.out[obase + oidx] = acc[r];
                        const T k0 = S.aux ? S.aux[obase + oidx] : T(0);
                        ech = fma(srow_line[hl + I], acc[r] - k0, ech);
                    } else if (MODE == M_POT) {
                        const T psi = acc[r];
                        if (S.aux) {
                            const T y = S.aux[vidx(I)] * psi;
                            if (S.out) S.out[obase + oidx] = y;
                            ech = fma(y, psi, ech);
                        }
                        if (RSM) {
                            if (S.rho) {
                                float2& q = rsm[I * LT + line];
                                FF f = first_orb ? FF{0.f, 0.f} : FF{q.x, q.y};
                                ff_add(f, (float)occ * (float)psi * (float)psi);
                                q = make_float2(f.hi, f.lo);
                            }
                        } else if (S.rho) {
                            racc[RSM ? 0 : cc][RSM ? 0 : r].add((T)occ * psi * psi);
                        }
                    }
                }
                if (MODE == M_KLAST || MODE == M_POT) e.add(ech);
            }
        }

        if ((MODE == M_POT && S.aux) || MODE == M_KLAST) {
            const double t = block_sum(e.get(), red);
            if (threadIdx.x == 0) S.part[(long long)orb * S.tiles + cur.tile] = t;
        }

        // M_POT: the unit ends -> flush its density
        if (MODE == M_POT && (!nxt.valid || nxt.unit != cur.unit)) {
            if (RSM && S.rho != nullptr && line_ok) {
                const long long grp = (cur.unit - S.blk0) / S.tiles;
                #pragma unroll 1
                for (int c = slot; c < nchunks; c += nslots)
                    #pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int I = c * R + r;
                        if (I >= n) continue;
                        const float2 q = rsm[I * LT + line];
                        const double v = (double)q.x + (double)q.y;
                        const long long oidx = vidx(I);
                        if (S.rho_gstride == 0) S.rho[oidx] += v;
                        else S.rho[grp * S.rho_gstride + oidx] = v;
                    }
            }
            if (!RSM && S.rho != nullptr && line_ok) {
                const long long grp = (cur.unit - S.blk0) / S.tiles;
                #pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    const int c = slot + cc * nslots;
                    #pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const int I = c * R + r;
                        if (c < nchunks && I < n) {
                            const long long oidx = vidx(I);
                            if (S.rho_gstride == 0) S.rho[oidx] += racc[RSM ? 0 : cc][RSM ? 0 : r].get();
                            else S.rho[grp * S.rho_gstride + oidx] = racc[RSM ? 0 : cc][RSM ? 0 : r].get();
                        }
                    }
                }
            }
            if (!RSM)
                #pragma unroll
                for (int cc = 0; cc < CPT; ++cc)
                    #pragma unroll
                    for (int r = 0; r < R; ++r) racc[RSM ? 0 : cc][RSM ? 0 : r].reset();
        }

        __syncthreads();   // buffer b is refilled by the next iteration's copies
        if (!nxt.valid) break;
        cur = nxt;
        b ^= 1;
    }
}

}  // namespace wvl
