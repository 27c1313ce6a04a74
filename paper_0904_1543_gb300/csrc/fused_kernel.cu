// The local Hamiltonian chain (Sec. "Local hamiltonian", Sec. "Three
// dimensional operators", Eqs. 3dconv and kinetic1d) as five kernels that keep
// fine-grid planes and column tiles on chip across several 1D filters.
//
// Every 3D operator of the chain (synthesis S, magic filter MF, its transpose
// MFT, the kinetic filter T = T_1 + T_2 + T_3, analysis A) is a product, or
// for T a sum, of 1D operators along the three axes, and 1D operators along
// different axes commute.  The chain therefore applies axis 3 in column
// kernels (tiles of all N3 rows x 32 FP32 / 16 FP64 columns at one I2) and
// axes 1 and 2 in plane kernels (one I3 plane), grouped so that what one
// kernel loads passes through several filters before it is written back.
// The wavelet transform is orthogonal along each axis (A_d S_d = identity,
// Eq. refinement with the orthogonality of h and g), so with a = S_3 c and
// s = S_1 S_2 a,
//   A T_3 s = A_3 T_3 A_1 A_2 S_1 S_2 a = A_3 T_3 a   and   <s, T_3 s> = <a, T_3 a>,
// and the analysis of the axis-3 kinetic term needs neither s nor A_1 A_2:
//
//   FZ_SYN3   (column)  a  = S_3 c                 c gathered from the compressed form
//   FZ_SKM12  (plane)   s  = S_1 S_2 a;  v = (T_1 + T_2) s;  t = MF_1 MF_2 s
//   FZ_POT3   (column)  psi_r = MF_3 t;  y_r = V psi_r;  rho += occ psi_r^2;  x = MFT_3 y_r
//   FZ_MFTA12 (plane)   w' = A_1 A_2 (MFT_1 MFT_2 x + v)
//   FZ_TA3    (column, two I2 rows)  H psi = A_3 (w' + T_3 a), written compressed
//
// which gives H psi = A (MFT V MF s + T s) (steps 1 to 7 of the chain),
// Ekin = <s, (T_1 + T_2) s> + <a, T_3 a> (partials from FZ_SKM12 and FZ_TA3)
// and Epot = <psi_r, V psi_r> (FZ_POT3).  Five round trips through HBM
// instead of the fifteen of the transposing passes: 52 instead of 140 bytes
// per orbital point in FP32.  The last kernel holds both I2 parities of its
// tile, so every coarse point's eight coefficients are on chip and the
// compressed form (scaling block, 7-component wavelet records) is written with
// consecutive lanes on consecutive addresses.
//
// Row pass: a lane owns one row (a warp, 32 rows at the same columns, so the
// periodic wrap is decided per warp) and 16 (or 8) consecutive outputs
// computed from a register window read as 16-byte vectors.  Column pass: a
// thread owns one 16-byte column vector and FZ_RC consecutive rows;
// consecutive threads take consecutive vectors of a row; wrapped rows come
// from a shared-memory offset table.  Taps are kernel parameters indexed at
// compile time, so the inner loops are loads and FMAs.  The plane row stride
// keeps an odd number of 16-byte words per row, so the 8 lanes of each phase
// of a lane-per-row vector load hit distinct banks.
#include <atomic>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

#include "pass_kernel.cuh"

namespace wvl {
namespace {

template <typename T>
struct Vec {
    T v[16 / sizeof(T)];
};

template <typename T>
__device__ __forceinline__ Vec<T> ldv(const T* p) {
    Vec<T> r;
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else {
        const double2 q = *reinterpret_cast<const double2*>(p);
        r.v[0] = q.x; r.v[1] = q.y;
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void stv(T* p, const T (&v)[16 / sizeof(T)]) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// compile-time loop: f(integral_constant<int, 0>) ... f(integral_constant<int, N - 1>),
// so tap indices are constants by construction (no run-time index or test)
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Energy accumulator of an energy partial (one CTA's share of Ekin): FP64
// in the FP64 form; in the FP32 form a compensated FP32 pair (two-sum,
// about 48 bits) of the item chains of at most 32 products, carried through
// the warp's shuffle tree and formed in FP64 from the warp on, as the
// potential kernel does for Epot -- FP64 additions through the tree took
// about 12 % of the last column kernel on GB300's narrow FP64 pipe.
template <typename T> struct EAcc;
template <> struct EAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double warp_sum() {
        double t = v;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        return t;
    }
};
template <> struct EAcc<float> {
    FF f{0.f, 0.f};
    __device__ __forceinline__ void add(float x) { ff_add(f, x); }
    __device__ __forceinline__ double warp_sum() {
        FF g = f;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, g.hi, o);
            const float ol = __shfl_down_sync(0xffffffffu, g.lo, o);
            ff_add(g, oh);
            g.lo += ol;
        }
        return (double)g.hi + (double)g.lo;
    }
};
// the CTA's sum: the warps' sums, then warp 0 adds them in a fixed tree
template <typename T>
__device__ __forceinline__ double fz_block_sum(EAcc<T>& e, double* red) {
    const double w = e.warp_sum();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5);
    if (lane == 0) red[warp] = w;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? red[lane] : 0.0;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            if (o < nw) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

// acc[k] += f[k & 1][t] win[j + D] for output k of a chunk whose window
// element j is input position (first output - HL + j).  FP32: outputs 2m,
// 2m + 1 take one packed FMA per window element, the element broadcast and
// the two taps a pair from tp (two FMAs per lane per instruction).
template <typename T, int KIND, int NOUT, int D, int NW>
__device__ __forceinline__ void fir(const T (&win)[NW], const T (&f)[2][32],
                                    const float2 (&tp)[32], T (&acc)[NOUT]) {
    constexpr int NT = KT<KIND>::NT;
    constexpr int W = NOUT + NT - 1 + KT<KIND>::EXTRA;
    if constexpr (sizeof(T) == 4) {
        static_assert(NOUT % 2 == 0, "output pairs");
        float2 a2[NOUT / 2];
        #pragma unroll
        for (int m = 0; m < NOUT / 2; ++m) a2[m] = make_float2(acc[2 * m], acc[2 * m + 1]);
        static_for<W>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const float2 ww = make_float2(win[j + D], win[j + D]);
            static_for<NOUT / 2>([&](auto mc) {
                constexpr int d = j - 2 * decltype(mc)::value;
                if constexpr (pair_on<KIND>(d))
                    a2[decltype(mc)::value] = __ffma2_rn(tp[d], ww, a2[decltype(mc)::value]);
            });
        });
        #pragma unroll
        for (int m = 0; m < NOUT / 2; ++m) {
            acc[2 * m] = a2[m].x;
            acc[2 * m + 1] = a2[m].y;
        }
    } else {
        static_for<W>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            static_for<NOUT>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int t = j - k - ((k & 1) ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
                if constexpr (tap_on<KIND>(t)) acc[k] = fma(f[k & 1][t], win[j + D], acc[k]);
            });
        });
    }
}

// WV 16-byte vectors of a periodic row from position p0 (a multiple of the
// vector width, possibly negative) into win, wrapped at ncols
template <typename T, int WV>
__device__ __forceinline__ void row_window(const T* __restrict__ row, int p0, int ncols,
                                           T (&win)[WV * (16 / sizeof(T))]) {
    constexpr int VEC = 16 / (int)sizeof(T);
    if (p0 >= 0 && p0 + WV * VEC <= ncols) {
        #pragma unroll
        for (int q = 0; q < WV; ++q) {
            const Vec<T> v = ldv(row + p0 + q * VEC);
            #pragma unroll
            for (int e = 0; e < VEC; ++e) win[q * VEC + e] = v.v[e];
        }
    } else {
        int pq = p0;
        while (pq < 0) pq += ncols;
        #pragma unroll
        for (int q = 0; q < WV; ++q) {
            const Vec<T> v = ldv(row + pq);
            #pragma unroll
            for (int e = 0; e < VEC; ++e) win[q * VEC + e] = v.v[e];
            pq += VEC;
            if (pq >= ncols) pq -= ncols;
        }
    }
}

// Row pass over a plane in shared memory:
//   dst(r, c) = sum_t f[c & 1][t] src(r, (c - HL + off(c & 1) + t) mod ncols)
// (the 1D filter of Eq. 1dconvtrans along the row, periodic)
template <typename T, int KIND, int RR>
__device__ __forceinline__ void row_pass_r(const T* __restrict__ src, T* __restrict__ dst,
                                           int nrows, int ncols, int RS, const T (&f)[2][32],
                                           const float2 (&tp)[32]) {
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int HL = KT<KIND>::HL;
    constexpr int HLR = (HL + VEC - 1) / VEC * VEC;   // window start, vector aligned
    constexpr int D = HLR - HL;
    constexpr int W = RR + KT<KIND>::NT - 1 + KT<KIND>::EXTRA;
    constexpr int WV = (W + D + VEC - 1) / VEC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    const int nrb = (nrows + 31) >> 5, nch = ncols / RR;
    #pragma unroll 1
    for (int it = warp; it < nrb * nch; it += nwarps) {
        const int ch = it / nrb, rb = it - ch * nrb;
        const int r = rb * 32 + lane;
        if (r >= nrows) continue;
        const int c0 = ch * RR;
        T win[WV * VEC];
        row_window<T, WV>(src + r * RS, c0 - HLR, ncols, win);
        T acc[RR];
        #pragma unroll
        for (int k = 0; k < RR; ++k) acc[k] = T(0);
        fir<T, KIND, RR, D>(win, f, tp, acc);
        T* o = dst + r * RS + c0;
        #pragma unroll
        for (int q = 0; q < RR / VEC; ++q) {
            T u[VEC];
            #pragma unroll
            for (int e = 0; e < VEC; ++e) u[e] = acc[q * VEC + e];
            stv(o + q * VEC, u);
        }
    }
}

// Row offsets of a periodic column: rowoff[FZ_PADR + q] = (q mod nrows) * RS
// for q in [-FZ_PADR, nrows + FZ_PADR), which covers every filter's window.
constexpr int FZ_PADR = 16;
__device__ __forceinline__ void fill_rowoff(int* rowoff, int nrows, int RS) {
    for (int q = (int)threadIdx.x - FZ_PADR; q < nrows + FZ_PADR; q += blockDim.x) {
        int w = q < 0 ? q + nrows : (q >= nrows ? q - nrows : q);
        rowoff[q + FZ_PADR] = w * RS;
    }
}

// 16 outputs per lane where the rows allow it (half the window loads and
// loop overhead per FMA of 8), else 8
template <typename T, int KIND>
__device__ __forceinline__ void row_pass(const T* __restrict__ src, T* __restrict__ dst,
                                         int nrows, int ncols, int RS, const T (&f)[2][32],
                                         const float2 (&tp)[32]) {
    if (ncols % 16 == 0) row_pass_r<T, KIND, 16>(src, dst, nrows, ncols, RS, f, tp);
    else row_pass_r<T, KIND, FZ_RR>(src, dst, nrows, ncols, RS, f, tp);
}

// FP32 row passes T_1 and MF_1 of the same plane from one window per chunk
// of 16 outputs: MF_1 src -> dst (shared memory), T_1 src -> vg (global, row
// stride ncols).  The kinetic window holds the magic filter's, so each
// filter's FMAs are those of its own row pass, in the same order.
template <typename T>
__device__ __forceinline__ void row_pass_kin_mf(const T* __restrict__ src, T* __restrict__ dst,
                                                T* __restrict__ vg, int nrows, int ncols, int RS,
                                                const FzParams<T>& p) {
    constexpr int RR = 16, VEC = 16 / (int)sizeof(T);
    constexpr int HLR = (KT<K_KIN>::HL + VEC - 1) / VEC * VEC;
    constexpr int DK = HLR - KT<K_KIN>::HL, DM = HLR - KT<K_MF>::HL;
    constexpr int WK = RR + KT<K_KIN>::NT - 1, WM = RR + KT<K_MF>::NT - 1;
    constexpr int WV = (WK + DK + VEC - 1) / VEC;
    static_assert(KT<K_KIN>::EXTRA == 0 && KT<K_MF>::EXTRA == 0 && DM >= 0 && WM + DM <= WV * VEC,
                  "the kinetic window holds the magic filter's");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    const int nrb = (nrows + 31) >> 5, nch = ncols / RR;
    #pragma unroll 1
    for (int it = warp; it < nrb * nch; it += nwarps) {
        const int ch = it / nrb, rb = it - ch * nrb;
        const int r = rb * 32 + lane;
        if (r >= nrows) continue;
        const int c0 = ch * RR;
        T win[WV * VEC];
        row_window<T, WV>(src + r * RS, c0 - HLR, ncols, win);
        T acc[RR];
        #pragma unroll
        for (int k = 0; k < RR; ++k) acc[k] = T(0);
        fir<T, K_KIN, RR, DK>(win, p.tap[1], p.tp[1], acc);
        T* const o = vg + (long long)r * ncols + c0;
        #pragma unroll
        for (int q = 0; q < RR / VEC; ++q) {
            T u[VEC];
            #pragma unroll
            for (int e = 0; e < VEC; ++e) u[e] = acc[q * VEC + e];
            stv(o + q * VEC, u);
        }
        #pragma unroll
        for (int k = 0; k < RR; ++k) acc[k] = T(0);
        fir<T, K_MF, RR, DM>(win, p.tap[3], p.tp[3], acc);
        T* const od = dst + r * RS + c0;
        #pragma unroll
        for (int q = 0; q < RR / VEC; ++q) {
            T u[VEC];
            #pragma unroll
            for (int e = 0; e < VEC; ++e) u[e] = acc[q * VEC + e];
            stv(od + q * VEC, u);
        }
    }
}

// One column-pass item: rows r0 .. r0 + FZ_RC - 1 of the 16-byte column
// vector cv,
//   acc[k][e] = sum_t f[k & 1][t] src((r0 + k - HL + off(k & 1) + t) mod nrows, cv VEC + e)
// the wrapped rows taken from the offset table (one path for every item)
template <typename T, int KIND, int RC = FZ_RC>
__device__ __forceinline__ void col_item(const T* __restrict__ src, const int* __restrict__ rowoff,
                                         int r0, int cv, const T (&f)[2][32],
                                         T (&acc)[RC][16 / sizeof(T)]) {
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int NT = KT<KIND>::NT, HL = KT<KIND>::HL;
    constexpr int W = RC + NT - 1 + KT<KIND>::EXTRA;
    static_assert(HL <= FZ_PADR && W - HL - RC <= FZ_PADR, "window beyond the offset table");
    #pragma unroll
    for (int k = 0; k < RC; ++k)
        #pragma unroll
        for (int e = 0; e < VEC; ++e) acc[k][e] = T(0);
    const T* base = src + cv * VEC;
    const int* ro = rowoff + FZ_PADR + r0 - HL;
    if constexpr (sizeof(T) == 4) {
        // FP32: the vector's two column pairs take one packed FMA each
        // (two FMAs per lane per instruction), which halves the FMA issue
        float2 a2[RC][2];
        #pragma unroll
        for (int k = 0; k < RC; ++k) a2[k][0] = a2[k][1] = make_float2(0.f, 0.f);
        static_for<W>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const float4 q = *reinterpret_cast<const float4*>(base + ro[j]);
            const float2 v01 = make_float2(q.x, q.y), v23 = make_float2(q.z, q.w);
            static_for<RC>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int t = j - k - ((k & 1) ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
                if constexpr (t >= KT<KIND>::SKIP && t < NT - KT<KIND>::SKIP) {
                    const float2 ff = make_float2(f[k & 1][t], f[k & 1][t]);
                    a2[k][0] = __ffma2_rn(ff, v01, a2[k][0]);
                    a2[k][1] = __ffma2_rn(ff, v23, a2[k][1]);
                }
            });
        });
        #pragma unroll
        for (int k = 0; k < RC; ++k) {
            acc[k][0] = a2[k][0].x;
            acc[k][1] = a2[k][0].y;
            acc[k][2] = a2[k][1].x;
            acc[k][3] = a2[k][1].y;
        }
    } else {
        static_for<W>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const Vec<T> v = ldv(base + ro[j]);
            static_for<RC>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int t = j - k - ((k & 1) ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
                if constexpr (t >= KT<KIND>::SKIP && t < NT - KT<KIND>::SKIP) {
                    #pragma unroll
                    for (int e = 0; e < VEC; ++e) acc[k][e] = fma(f[k & 1][t], v.v[e], acc[k][e]);
                }
            });
        });
    }
}

// ------------------------------------------------------------ plane kernels
// threads of a column kernel: FZ_TA3 holds two I2 rows per job
template <int PROG>
__host__ __device__ constexpr int fz_cthreads() { return PROG == FZ_TA3 ? 2 * FZ_CTHREADS : FZ_CTHREADS; }

template <typename T, int PROG>
__global__ void __launch_bounds__(FZ_PTHREADS)
fz_plane_kernel(const __grid_constant__ FzParams<T> p) {
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int RC = FZ_RC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[FZ_PTHREADS / 32];
    __shared__ int rowoff[FZ_MAX_FINE + 2 * FZ_PADR];
    const long long job = blockIdx.x;
    int si = 0;
    #pragma unroll 1
    while (si + 1 < p.nseg && job >= p.seg[si + 1].blk0) ++si;
    const FzSeg<T>& S = p.seg[si];
    const long long loc = job - S.blk0;
    const int I3 = (int)(loc % S.N3);
    const int o = (int)(loc / S.N3);
    const int N1 = S.N1, N2 = S.N2, RS = S.RS;
    const long long pbase = (long long)o * S.P + (long long)I3 * N1 * N2;
    T* const X = reinterpret_cast<T*>(smem_raw);
    T* const Y = X + N2 * RS;
    const int ncv = N1 / VEC;
    const int nitems = (N2 / RC) * ncv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NWARP = FZ_PTHREADS / 32;

    // the plane, row I2 -> X + I2 RS (a warp per row, lanes over its vectors)
    {
        const T* src = S.in + pbase;
        #pragma unroll 1
        for (int r = warp; r < N2; r += NWARP)
            for (int c = lane; c < ncv; c += 32)
                cp_async16(X + r * RS + c * VEC, src + (long long)r * N1 + c * VEC);
        cp_commit();
        fill_rowoff(rowoff, N2, RS);
        cp_wait<0>();
        __syncthreads();
    }

    if constexpr (PROG == FZ_SKM12) {
        EAcc<T> e;
        // s = S_1 S_2 a -> X: the column pass (S_2) first, then the row pass
        // (the two commute; this order measured 1 % faster)
        #pragma unroll 1
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
            T acc[RC][VEC];
            col_item<T, K_SYN>(X, rowoff, r0, cv, p.tap[0], acc);
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk) stv(Y + (r0 + kk) * RS + cv * VEC, acc[kk]);
        }
        __syncthreads();
        row_pass<T, K_SYN>(Y, X, N2, N1, RS, p.tap[0], p.tp[0]);
        __syncthreads();
        if (sizeof(T) == 4 && N1 % 16 == 0 && S.part != nullptr && S.out2 != nullptr) {
            // H psi, FP32: T_1 s -> v and MF_1 s -> Y in one row pass (one
            // window per chunk, two fewer phases); then per column item
            // t = MF_2 Y and v += T_2 s with the Ekin part <s, v>, the same
            // operations in the same order as the phases below (bit-identical
            // results; 1.414 -> 1.404 ms per headline step for SYN3 + SKM12).
            // The FP32 kernel fits 128 registers (two CTAs per SM).
            T* const vg = S.out2 + pbase;
            row_pass_kin_mf<T>(X, Y, vg, N2, N1, RS, p);
            __syncthreads();
            #pragma unroll 1
            for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
                const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
                T acc[RC][VEC];
                col_item<T, K_MF>(Y, rowoff, r0, cv, p.tap[3], acc);
                #pragma unroll
                for (int kk = 0; kk < RC; ++kk)
                    stv(S.out3 + pbase + (long long)(r0 + kk) * N1 + cv * VEC, acc[kk]);
                Vec<T> t1[RC];
                #pragma unroll
                for (int kk = 0; kk < RC; ++kk) t1[kk] = ldv(vg + (long long)(r0 + kk) * N1 + cv * VEC);
                col_item<T, K_KIN>(X, rowoff, r0, cv, p.tap[2], acc);
                T ei = T(0);
                #pragma unroll
                for (int kk = 0; kk < RC; ++kk) {
                    const Vec<T> sv = ldv(X + (r0 + kk) * RS + cv * VEC);
                    T v[VEC];
                    #pragma unroll
                    for (int q = 0; q < VEC; ++q) {
                        v[q] = acc[kk][q] + t1[kk].v[q];
                        ei = fma(sv.v[q], v[q], ei);
                    }
                    stv(vg + (long long)(r0 + kk) * N1 + cv * VEC, v);
                }
                e.add(ei);
            }
            const double tot = fz_block_sum(e, red);
            if (threadIdx.x == 0) S.part[(long long)o * S.ptiles + S.poff + I3] = tot;
            return;
        }
        // v = T_1 s + T_2 s, Ekin part <s, v> (not for the density alone;
        // v stored for H psi only)
        if (S.part != nullptr) {
        row_pass<T, K_KIN>(X, Y, N2, N1, RS, p.tap[1], p.tp[1]);
        __syncthreads();
        #pragma unroll 1
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
            T acc[RC][VEC];
            col_item<T, K_KIN>(X, rowoff, r0, cv, p.tap[2], acc);
            T ei = T(0);   // the item's <s, v> (at most 32 products), then added in FP64
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk) {
                const int off = (r0 + kk) * RS + cv * VEC;
                const Vec<T> t1 = ldv(Y + off);
                const Vec<T> sv = ldv(X + off);
                T v[VEC];
                #pragma unroll
                for (int q = 0; q < VEC; ++q) {
                    v[q] = acc[kk][q] + t1.v[q];
                    ei = fma(sv.v[q], v[q], ei);
                }
                if (S.out2 != nullptr) stv(S.out2 + pbase + (long long)(r0 + kk) * N1 + cv * VEC, v);
            }
            e.add(ei);
        }
        __syncthreads();
        }
        // t = MF_1 MF_2 s
        row_pass<T, K_MF>(X, Y, N2, N1, RS, p.tap[3], p.tp[3]);
        __syncthreads();
        #pragma unroll 1
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
            T acc[RC][VEC];
            col_item<T, K_MF>(Y, rowoff, r0, cv, p.tap[3], acc);
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk)
                stv(S.out3 + pbase + (long long)(r0 + kk) * N1 + cv * VEC, acc[kk]);
        }
        if (S.part != nullptr) {
            const double tot = fz_block_sum(e, red);
            if (threadIdx.x == 0) S.part[(long long)o * S.ptiles + S.poff + I3] = tot;
        }
    } else {
        // FZ_MFTA12: w = MFT_1 MFT_2 x + v, then w' = A_1 A_2 w
        row_pass<T, K_MFT>(X, Y, N2, N1, RS, p.tap[0], p.tp[0]);
        __syncthreads();
        // X is free: each thread fetches the v of its own outputs there,
        // overlapped with its column passes, and leaves w in its place
        #pragma unroll 1
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk)
                cp_async16(X + (r0 + kk) * RS + cv * VEC,
                           S.in2 + pbase + (long long)(r0 + kk) * N1 + cv * VEC);
        }
        cp_commit();
        #pragma unroll 1
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
            T acc[RC][VEC];
            col_item<T, K_MFT>(Y, rowoff, r0, cv, p.tap[0], acc);
            cp_wait<0>();
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk) {
                T* const xw = X + (r0 + kk) * RS + cv * VEC;
                const Vec<T> v = ldv(xw);
                T w[VEC];
                #pragma unroll
                for (int q = 0; q < VEC; ++q) w[q] = acc[kk][q] + v.v[q];
                stv(xw, w);
            }
        }
        __syncthreads();
        row_pass<T, K_ANA>(X, Y, N2, N1, RS, p.tap[1], p.tp[1]);
        __syncthreads();
        #pragma unroll 1
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int k = it / ncv, cv = it - k * ncv, r0 = k * RC;
            T acc[RC][VEC];
            col_item<T, K_ANA>(Y, rowoff, r0, cv, p.tap[1], acc);
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk)
                stv(S.out + pbase + (long long)(r0 + kk) * N1 + cv * VEC, acc[kk]);
        }
    }
}

// ----------------------------------------------------------- column kernels
// A tile is N3 rows (I3) of LTC = 128 bytes of columns (I1 from c0) at one I2
// (FZ_TA3: at I2 = 2 i2 and 2 i2 + 1, one sub-tile each); column-pass item it
// covers rows 8 (it / 8) .. + 7 of column vector it % 8 of a sub-tile
// (vectors past a partial last tile are idle).
// CTAs per SM the register allocation must allow
template <int PROG>
__host__ __device__ constexpr int fz_cminb() { return PROG == FZ_SYN3 || PROG == FZ_POT3 ? 4 : 3; }

template <typename T, int PROG>
__global__ void __launch_bounds__(fz_cthreads<PROG>(), fz_cminb<PROG>())
fz_col_kernel(const __grid_constant__ FzParams<T> p) {
    constexpr int VEC = 16 / (int)sizeof(T);
    constexpr int RC = FZ_RC;
    constexpr int LTC = fz_ltc<T>();
    constexpr int CV = LTC / VEC;        // 8 column vectors per tile row
    constexpr int NT = fz_cthreads<PROG>();
    static_assert(CV == 8, "tile rows are 128 bytes");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    __shared__ int rowoff[FZ_MAX_FINE + 2 * FZ_PADR];
    const long long job = blockIdx.x;
    int si = 0;
    #pragma unroll 1
    while (si + 1 < p.nseg && job >= p.seg[si + 1].blk0) ++si;
    const FzSeg<T>& S = p.seg[si];
    const long long loc = job - S.blk0;
    constexpr int NSUB = PROG == FZ_TA3 ? 2 : 1;   // I2 rows per job
    const int cb = (int)(loc % S.ncb);
    const long long rest = loc / S.ncb;
    const int I2 = (int)(rest % (S.N2 / NSUB)) * NSUB;
    const int u = (int)(rest / (S.N2 / NSUB));   // orbital, or orbital group for FZ_POT3
    const int N1 = S.N1, N2 = S.N2, N3 = S.N3, RS = S.RS;
    const long long plane = (long long)N1 * N2;
    const int c0 = cb * LTC;
    const int ncv = min(LTC, N1 - c0) / VEC;
    const long long col0 = (long long)I2 * N1 + c0;   // (I3 = 0, I2, c0) in an orbital
    T* const X = reinterpret_cast<T*>(smem_raw);
    T* const Y = X + NSUB * N3 * RS;
    const int nitems = (N3 / RC) * CV;   // per sub-tile
    const int ptile = (I2 / NSUB) * S.ncb + cb;
    fill_rowoff(rowoff, N3, RS);

    // tile rows (ncv vectors each) of sub-tiles 0 .. NSUB-1 -> dst + (sub N3 + I3) RS;
    // thread t copies vector t % 8 of rows t / 8, t / 8 + NT / 8, ...
    auto load_tile = [&](T* dst, const T* src) {
        const int c = threadIdx.x & (CV - 1);
        if (c < ncv)
            #pragma unroll 1
            for (int r = threadIdx.x / CV; r < NSUB * N3; r += NT / CV) {
                const int sub = r >= N3, rr = r - sub * N3;
                cp_async16(dst + r * RS + c * VEC, src + sub * N1 + (long long)rr * plane + c * VEC);
            }
        cp_commit();
    };

    if constexpr (PROG == FZ_SYN3) {
        // gather: tile element (I3, I1) is c^mu at coarse point
        // (I1/2, I2/2, I3/2), mu = a1 + 2 a2 + 4 a3 (the interleaved layout).
        // The job walks the orbitals of group u on this tile; the next
        // orbital's gather goes into the other buffer while this one is
        // filtered
        const int ncols = ncv * VEC;
        const int a2 = 2 * (I2 & 1);
        const int x = threadIdx.x & (LTC - 1);
        const int I1 = c0 + x;
        const long long cxy = (long long)(I2 >> 1) * S.n1 + (I1 >> 1);
        const long long nxy = (long long)S.n2 * S.n1;
        // the thread's rows rg, rg + RSTEP, ... share the parity of rg (RSTEP
        // is even), so mu is fixed and the source advances by RSTEP / 2 coarse
        // planes per row: one pointer step per element
        constexpr int RSTEP = NT / LTC;
        static_assert(RSTEP % 2 == 0, "rows of one parity per thread");
        const int rg = threadIdx.x / LTC;
        const int mu = (I1 & 1) + a2 + 4 * (rg & 1);
        const long long ci0 = (long long)(rg >> 1) * nxy + cxy;
        const long long soff = (mu == 0) ? ci0 : S.P / 8 + ci0 * 7 + mu - 1;
        const long long step = (mu == 0 ? 1 : 7) * (RSTEP / 2) * nxy;
        auto gather = [&](T* dst, int o) {
            const T* src = S.in + (long long)o * S.P + soff;
            if (x < ncols)
                #pragma unroll 1
                for (int r = rg; r < N3; r += RSTEP, src += step) cp_async(dst + r * RS + x, src);
            cp_commit();
        };
        const int o0 = u * S.opg, o1 = min(S.norb, o0 + S.opg);
        gather(X, o0);
        #pragma unroll 1
        for (int o = o0; o < o1; ++o) {
            T* const cur = ((o - o0) & 1) ? Y : X;
            cp_wait<0>();
            __syncthreads();   // every thread also left the previous orbital's buffer
            if (o + 1 < o1) gather(((o - o0) & 1) ? X : Y, o + 1);
            T* const ob = S.out + (long long)o * S.P + col0;
            #pragma unroll 1
            for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
                const int k = it >> 3, cv = it & 7, r0 = k * RC;
                if (cv >= ncv) continue;
                T acc[RC][VEC];
                col_item<T, K_SYN>(cur, rowoff, r0, cv, p.tap[0], acc);
                #pragma unroll
                for (int kk = 0; kk < RC; ++kk) stv(ob + (long long)(r0 + kk) * plane + cv * VEC, acc[kk]);
            }
        }
    } else if constexpr (PROG == FZ_TA3) {
        // H psi = A_3 (w' + T_3 a) on both I2 rows; Ekin part <a, T_3 a>
        // (the energy alone when there is no w')
        const bool full = S.in != nullptr;
        const long long ob = (long long)u * S.P + col0;
        // a first, then w' in a second copy group: T_3 a runs while w' is
        // still arriving (0.606 -> 0.592 ms per headline step).  Tiles have
        // at most FZ_MAX_FINE rows, so a thread has at most one item.
        static_assert(NSUB * (FZ_MAX_FINE / RC) * CV <= NT, "one item per thread");
        load_tile(Y, S.in2 + ob);             // a
        if (full) load_tile(X, S.in + ob);    // w'
        if (full) cp_wait<1>();
        else cp_wait<0>();
        __syncthreads();
        EAcc<T> e;
        {
            const int it = threadIdx.x;
            const int sub = it >= nitems, r = it - sub * nitems;
            const int k = r >> 3, cv = r & 7, r0 = k * RC;
            const bool has = it < NSUB * nitems && cv < ncv;
            const int so = sub * N3 * RS;
            T acc[RC][VEC];
            if (has) col_item<T, K_KIN>(Y + so, rowoff, r0, cv, p.tap[0], acc);
            if (full) {
                cp_wait<0>();
                __syncthreads();
            }
            if (has) {
                T ei = T(0);
                #pragma unroll
                for (int kk = 0; kk < RC; ++kk) {
                    const int off = so + (r0 + kk) * RS + cv * VEC;
                    const Vec<T> av = ldv(Y + off);
                    #pragma unroll
                    for (int q = 0; q < VEC; ++q) ei = fma(av.v[q], acc[kk][q], ei);
                    if (full) {
                        const Vec<T> wv = ldv(X + off);
                        T z[VEC];
                        #pragma unroll
                        for (int q = 0; q < VEC; ++q) z[q] = wv.v[q] + acc[kk][q];
                        stv(X + off, z);
                    }
                }
                e.add(ei);
            }
        }
        __syncthreads();
        if (full) {
        // A_3 z -> Y (a is no longer needed)
        #pragma unroll 1
        for (int it = threadIdx.x; it < NSUB * nitems; it += blockDim.x) {
            const int sub = it >= nitems, r = it - sub * nitems;
            const int k = r >> 3, cv = r & 7, r0 = k * RC;
            if (cv >= ncv) continue;
            const int so = sub * N3 * RS;
            T acc[RC][VEC];
            col_item<T, K_ANA>(X + so, rowoff, r0, cv, p.tap[1], acc);
            #pragma unroll
            for (int kk = 0; kk < RC; ++kk) stv(Y + so + (r0 + kk) * RS + cv * VEC, acc[kk]);
        }
        __syncthreads();
        // compressed form of the tile's coarse points (i1 from c0 / 2, i2, every
        // i3): per i3 a run of 7 nci wavelet coefficients (records of the
        // components mu = 1..7) and a run of nci scaling coefficients, both
        // 16-byte aligned; lane g of a warp writes 16-byte group g of the
        // two runs (the wavelet run first), reading its elements from Y at
        // offsets that depend on g only
        {
            T* const cc = S.out + (long long)u * S.P;
            T* const cf = cc + S.P / 8;
            const int nci = ncv * VEC / 2;                 // coarse points of the tile row
            // the adjoint of E_loc: H psi scaled by 2 occ g
            const T osc = S.gscale != nullptr ? T(2.0 * S.occ[u] * S.gscale[0]) : T(1);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const long long kb = (long long)(I2 >> 1) * S.n1 + (c0 >> 1);
            const long long nxy = (long long)S.n2 * S.n1;
            const int ngw = 7 * nci / VEC, ngs = nci / VEC;   // 16-byte groups of the runs
            const bool wav = lane < ngw, act = lane < ngw + ngs;
            // element pos of the wavelet run is record position 7 i1 + mu - 1
            // (mu = a1 + 2 a2 + 4 a3) of coarse point i1, at Y offset
            // a2 N3 RS + a3 RS + 2 i1 + a1 from the tile's (a3 = 0) row 2 i3;
            // element pos of the scaling run is coarse point pos (mu = 0)
            int yo[VEC];
            #pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int pos = (wav ? lane : lane - ngw) * VEC + q;
                const int i1 = pos / 7, mu = pos - 7 * i1 + 1;
                yo[q] = wav ? (mu >> 1 & 1) * N3 * RS + (mu >> 2) * RS + 2 * i1 + (mu & 1) : 2 * pos;
            }
            if (act)
                #pragma unroll 1
                for (int i3 = warp; i3 < N3 / 2; i3 += NT / 32) {
                    const long long k0 = (long long)i3 * nxy + kb;
                    const T* const y0 = Y + (2 * i3) * RS;
                    T v[VEC];
                    #pragma unroll
                    for (int q = 0; q < VEC; ++q) v[q] = y0[yo[q]] * osc;
                    stv(wav ? cf + 7 * k0 + lane * VEC : cc + k0 + (lane - ngw) * VEC, v);
                }
        }
        }
        const double tot = fz_block_sum(e, red);
        if (threadIdx.x == 0) S.part[(long long)u * S.ptiles + S.poff + ptile] = tot;
    } else {
        // FZ_POT3: the orbitals of group u in order; each thread owns one
        // item, so its density sums stay in registers across the orbitals;
        // the potential tile is staged once per job.  An item is RP rows of
        // a 16-byte column vector: N3 / 16 rows where N3 is a multiple of 16
        // from 64 up (FP32), so that the N3 / RP x 8 items fill the CTA's 128
        // threads (8 rows: 80 and 96 of them busy on 80- and 96-row tiles);
        // else 8 (the magic filter and its transpose take the same taps for
        // both output parities, so any RP works)
        auto pot3 = [&](auto rpc) {
            constexpr int RP = decltype(rpc)::value;
            T* const Z = Y + N3 * RS;
            const int o0 = u * S.opg, o1 = min(S.norb, o0 + S.opg);
            // Epot partial of orbital o0 + j from warp w: epw[(j % FZ_EPW) * 4 + w]
            // (FP32: the compensated pair, epf), written out every FZ_EPW
            // orbitals; occf holds the FP32 occupations of the current FZ_EPW
            constexpr int NW = NT / 32;
            double* const epw = reinterpret_cast<double*>(Z + N3 * RS);
            [[maybe_unused]] float2* const epf = reinterpret_cast<float2*>(epw);
            [[maybe_unused]] float* const occf = reinterpret_cast<float*>(epw + FZ_EPW * NW);
            const int k = (int)threadIdx.x >> 3, cv = (int)threadIdx.x & 7, r0 = k * RP;
            const bool mine = (int)threadIdx.x < (N3 / RP) * CV && cv < ncv;
            constexpr bool PK = sizeof(T) == 4;   // FP32: compensated pairs, two columns at once
            [[maybe_unused]] FF2 rp[PK ? RP : 1][PK ? 2 : 1];
            [[maybe_unused]] RhoAcc<T> racc[PK ? 1 : RP][PK ? 1 : VEC];
            const bool pot = S.V != nullptr, full = S.out != nullptr;
            if (pot) load_tile(Z, S.V + col0);
            load_tile(X, S.in + (long long)o0 * S.P + col0);
            #pragma unroll 1
            for (int o = o0; o < o1; ++o) {
                const int j = (o - o0) % FZ_EPW;
                if constexpr (PK) {
                    // the occupations of the next FZ_EPW orbitals as floats, so
                    // that the orbital loop itself runs no FP64 instruction
                    if (j == 0 && (int)threadIdx.x < min(FZ_EPW, o1 - o))
                        occf[threadIdx.x] = (float)(S.occ ? S.occ[o + threadIdx.x] : 1.0);
                }
                cp_wait<0>();
                __syncthreads();
                T ei = T(0);   // this thread's Epot terms of the orbital (at most 32 products)
                T occ;
                if constexpr (PK) occ = occf[j];
                else occ = (T)(S.occ ? S.occ[o] : 1.0);
                T acc[RP][VEC];
                if (mine) {
                    col_item<T, K_MF, RP>(X, rowoff, r0, cv, p.tap[0], acc);
                    if constexpr (PK) {
                        const float2 oc = make_float2(occ, occ);
                        #pragma unroll
                        for (int kk = 0; kk < RP; ++kk) {
                            const float2 a01 = make_float2(acc[kk][0], acc[kk][1]);
                            const float2 a23 = make_float2(acc[kk][2], acc[kk][3]);
                            ff2_add(rp[kk][0], __fmul2_rn(__fmul2_rn(oc, a01), a01));
                            ff2_add(rp[kk][1], __fmul2_rn(__fmul2_rn(oc, a23), a23));
                        }
                    } else {
                        #pragma unroll
                        for (int kk = 0; kk < RP; ++kk)
                            #pragma unroll
                            for (int q = 0; q < VEC; ++q) racc[kk][q].add(occ * acc[kk][q] * acc[kk][q]);
                    }
                    #pragma unroll
                    for (int kk = 0; kk < RP; ++kk) {
                        const int off = (r0 + kk) * RS + cv * VEC;
                        if (pot) {
                            const Vec<T> vv = ldv(Z + off);
                            T y[VEC];
                            #pragma unroll
                            for (int q = 0; q < VEC; ++q) {
                                y[q] = vv.v[q] * acc[kk][q];
                                ei = fma(y[q], acc[kk][q], ei);
                            }
                            if (full) stv(Y + off, y);
                        }
                    }
                }
                __syncthreads();
                // X is free: fetch the next orbital's tile during the MFT pass
                if (o + 1 < o1) load_tile(X, S.in + (long long)(o + 1) * S.P + col0);
                if (mine && full) {
                    col_item<T, K_MFT, RP>(Y, rowoff, r0, cv, p.tap[1], acc);
                    T* const ob = S.out + (long long)o * S.P + col0;
                    #pragma unroll
                    for (int kk = 0; kk < RP; ++kk) stv(ob + (long long)(r0 + kk) * plane + cv * VEC, acc[kk]);
                }
                // the warp's sum of the threads' terms: FP64 in the FP64 form; in the
                // FP32 form a compensated FP32 pair (about 48 bits) through the
                // shuffle tree, kept as a pair until the flush adds the warps' pairs
                // in FP64 (a tree of FP64 additions per orbital kept the FP64 pipe
                // of GB300 80 % busy; converting each warp's pair per orbital cost
                // 0.007 ms per headline step against converting at the flush)
                if constexpr (PK) {
                    FF f{ei, 0.f};
                    #pragma unroll
                    for (int sh = 16; sh > 0; sh >>= 1) {
                        const float oh = __shfl_down_sync(0xffffffffu, f.hi, sh);
                        const float ol = __shfl_down_sync(0xffffffffu, f.lo, sh);
                        ff_add(f, oh);
                        f.lo += ol;
                    }
                    if ((threadIdx.x & 31) == 0) epf[j * NW + (threadIdx.x >> 5)] = make_float2(f.hi, f.lo);
                } else {
                    double ew = ei;
                    #pragma unroll
                    for (int sh = 16; sh > 0; sh >>= 1) ew += __shfl_down_sync(0xffffffffu, ew, sh);
                    if ((threadIdx.x & 31) == 0) epw[j * NW + (threadIdx.x >> 5)] = ew;
                }
                if (j == FZ_EPW - 1 || o + 1 == o1) {
                    // orbitals o - j .. o: warp partials in a fixed order
                    __syncthreads();
                    if ((int)threadIdx.x <= j && S.part != nullptr) {
                        double t = 0.0;
                        #pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            double ew;
                            if constexpr (PK) {
                                const float2 e = epf[threadIdx.x * NW + w];
                                ew = (double)e.x + (double)e.y;
                            } else {
                                ew = epw[threadIdx.x * NW + w];
                            }
                            t += ew;
                        }
                        S.part[(long long)(o - j + (int)threadIdx.x) * S.ptiles + S.poff + ptile] = t;
                    }
                }
            }
            if (mine && S.rho != nullptr) {
                double* const rb = S.rho + (long long)u * S.rho_gstride;
                #pragma unroll
                for (int kk = 0; kk < RP; ++kk)
                    #pragma unroll
                    for (int q = 0; q < VEC; ++q) {
                        const long long g = (long long)(r0 + kk) * plane + col0 + cv * VEC + q;
                        double v;
                        if constexpr (PK) v = ff2_get(rp[kk][q >> 1], q & 1);
                        else v = racc[kk][q].get();
                        if (S.rho_gstride == 0) rb[g] += v;
                        else rb[g] = v;
                    }
            }
        };
        const int rp = (sizeof(T) == 4 && N3 % 16 == 0 && N3 >= 64) ? N3 / 16 : FZ_RC;
        if (rp == 4) pot3(std::integral_constant<int, 4>{});
        else if (rp == 5) pot3(std::integral_constant<int, 5>{});
        else if (rp == 6) pot3(std::integral_constant<int, 6>{});
        else if (rp == 7) pot3(std::integral_constant<int, 7>{});
        else pot3(std::integral_constant<int, FZ_RC>{});
    }
}

// ------------------------------------------------------------------ host
template <int PROG>
constexpr bool fz_is_plane() { return PROG == FZ_SKM12 || PROG == FZ_MFTA12; }

constexpr int FZ_SMEM_OPTIN = 224 * 1024;   // under the opt-in limit with the static reduction buffer

template <typename T, int PROG>
cudaError_t fz_ensure_attr() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        if constexpr (fz_is_plane<PROG>())
            err = cudaFuncSetAttribute(fz_plane_kernel<T, PROG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, FZ_SMEM_OPTIN);
        else
            err = cudaFuncSetAttribute(fz_col_kernel<T, PROG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, FZ_SMEM_OPTIN);
        if (err != cudaSuccess) return err;
        done.fetch_or(bit);
    }
    return cudaSuccess;
}

template <typename T, int PROG>
cudaError_t fz_launch(const FzParams<T>& p, size_t smem, cudaStream_t st) {
    cudaError_t err = fz_ensure_attr<T, PROG>();
    if (err != cudaSuccess) return err;
    if (p.njobs <= 0) return cudaSuccess;
    if (p.njobs > 0x7fffffffLL || smem > (size_t)FZ_SMEM_OPTIN) return cudaErrorInvalidConfiguration;
    if constexpr (fz_is_plane<PROG>() && sizeof(T) == 4) {
        // the row passes' tap pairs (the slots and filters of the row passes
        // in fz_plane_kernel)
        FzParams<T> q = p;
        if constexpr (PROG == FZ_SKM12) {
            tap_pairs<K_SYN>(q.tap[0], q.tp[0]);
            tap_pairs<K_KIN>(q.tap[1], q.tp[1]);
            tap_pairs<K_MF>(q.tap[3], q.tp[3]);
        } else {
            tap_pairs<K_MFT>(q.tap[0], q.tp[0]);
            tap_pairs<K_ANA>(q.tap[1], q.tp[1]);
        }
        fz_plane_kernel<T, PROG><<<dim3((unsigned)p.njobs), dim3(FZ_PTHREADS), smem, st>>>(q);
    } else if constexpr (fz_is_plane<PROG>())
        fz_plane_kernel<T, PROG><<<dim3((unsigned)p.njobs), dim3(FZ_PTHREADS), smem, st>>>(p);
    else
        fz_col_kernel<T, PROG><<<dim3((unsigned)p.njobs), dim3(fz_cthreads<PROG>()), smem, st>>>(p);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
size_t fz_smem(int prog, int N1, int N2, int N3) {
    if (prog == FZ_SKM12 || prog == FZ_MFTA12)
        return 2 * (size_t)N2 * fz_plane_rs<T>(N1) * sizeof(T);
    // FZ_POT3 also stages the potential tile and keeps per-warp Epot partials
    // and FP32 occupations;
    // FZ_TA3 holds two sub-tiles in each of its two buffers
    if (prog == FZ_POT3)
        return 3 * (size_t)N3 * fz_ltc<T>() * sizeof(T) + (size_t)FZ_EPW * (FZ_CTHREADS / 32) * 8 +
               (size_t)FZ_EPW * sizeof(float);
    if (prog == FZ_TA3) return 4 * (size_t)N3 * fz_ltc<T>() * sizeof(T);
    return 2 * (size_t)N3 * fz_ltc<T>() * sizeof(T);
}

template <typename T>
cudaError_t launch_fused(int prog, const FzParams<T>& p, size_t smem, cudaStream_t st) {
    switch (prog) {
    case FZ_SYN3: return fz_launch<T, FZ_SYN3>(p, smem, st);
    case FZ_SKM12: return fz_launch<T, FZ_SKM12>(p, smem, st);
    case FZ_POT3: return fz_launch<T, FZ_POT3>(p, smem, st);
    case FZ_MFTA12: return fz_launch<T, FZ_MFTA12>(p, smem, st);
    case FZ_TA3: return fz_launch<T, FZ_TA3>(p, smem, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t prepare_fused_kernels() {
    cudaError_t e;
    if ((e = fz_ensure_attr<T, FZ_SYN3>()) != cudaSuccess) return e;
    if ((e = fz_ensure_attr<T, FZ_SKM12>()) != cudaSuccess) return e;
    if ((e = fz_ensure_attr<T, FZ_POT3>()) != cudaSuccess) return e;
    if ((e = fz_ensure_attr<T, FZ_MFTA12>()) != cudaSuccess) return e;
    return fz_ensure_attr<T, FZ_TA3>();
}

template size_t fz_smem<float>(int, int, int, int);
template size_t fz_smem<double>(int, int, int, int);
template cudaError_t launch_fused<float>(int, const FzParams<float>&, size_t, cudaStream_t);
template cudaError_t launch_fused<double>(int, const FzParams<double>&, size_t, cudaStream_t);
template cudaError_t prepare_fused_kernels<float>();
template cudaError_t prepare_fused_kernels<double>();

}  // namespace wvl
