// The 1D "convolve + transpose" pass (Eqs. 1dconvtrans, kinetic1d) for
// sm_103a, templated on the element type, the operator, the epilogue and the
// number of consecutive outputs per thread.
//
// A CTA owns a tile of LT consecutive lines of one orbital and keeps the
// whole periodic lines in shared memory, extended by the left/right halos
// (wrapped while staging, which is how the periodic boundary is applied).  A
// thread computes R consecutive outputs of one line from a register window of
// R + NT - 1 (+1 for the two-phase wavelet filters) shared-memory values; taps
// are kernel parameters (constant bank) and indices are compile-time, so the
// inner loop is loads and FMAs only.  Outputs go to F[I][a] with the line index
// fastest, so each warp's stores are coalesced (LT contiguous elements).
#pragma once
#include <cuda_runtime.h>

#include "wvl_internal.h"

namespace wvl {

template <int KIND> struct KT;
template <> struct KT<K_MF>  { static constexpr int NT = 16, OFF0 = 0, OFF1 = 0, EXTRA = 0; };
template <> struct KT<K_MFT> { static constexpr int NT = 16, OFF0 = 0, OFF1 = 0, EXTRA = 0; };
template <> struct KT<K_KIN> { static constexpr int NT = 29, OFF0 = 0, OFF1 = 0, EXTRA = 0; };
template <> struct KT<K_SYN> { static constexpr int NT = 16, OFF0 = 0, OFF1 = 1, EXTRA = 1; };
template <> struct KT<K_ANA> { static constexpr int NT = 16, OFF0 = 1, OFF1 = 0, EXTRA = 1; };

// compensated single-precision accumulation (Knuth two-sum)
struct FF { float hi, lo; };
__device__ __forceinline__ void ff_add(FF& a, float x) {
    float s = a.hi + x;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (x - bb);
    a.hi = s;
    a.lo += e;
}

template <typename T> struct Acc;
template <> struct Acc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void fma_add(double a, double b) { v = fma(a, b, v); }
    __device__ __forceinline__ double get() const { return v; }
    __device__ __forceinline__ void reset() { v = 0.0; }
};
template <> struct Acc<float> {
    FF f{0.f, 0.f};
    __device__ __forceinline__ void add(float x) { ff_add(f, x); }
    __device__ __forceinline__ void fma_add(float a, float b) { ff_add(f, a * b); }
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
        for (int w = 0; w < NTHREADS / 32; ++w) t += red[w];
    }
    __syncthreads();
    return t;
}

// R outputs of one line from the shared-memory row (srow[j] <-> position
// i0 - HL + j); acc must hold the initial values.
template <typename T, int KIND, int R>
__device__ __forceinline__ void conv_chunk(const T* __restrict__ srow,
                                           const PassParams<T>& p, T (&acc)[R]) {
    constexpr int NT = KT<KIND>::NT;
    constexpr int W = R + NT - 1 + KT<KIND>::EXTRA;
    #pragma unroll
    for (int j = 0; j < W; ++j) {
        const T v = srow[j];
        #pragma unroll
        for (int r = 0; r < R; ++r) {
            const int t = j - r - ((r & 1) ? KT<KIND>::OFF1 : KT<KIND>::OFF0);
            if (t >= 0 && t < NT) acc[r] = fma(p.f[r & 1][t], v, acc[r]);
        }
    }
}

template <typename T, int KIND, int MODE, int R>
__global__ void __launch_bounds__(NTHREADS)
pass_kernel(const __grid_constant__ PassParams<T> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[NTHREADS / 32];

    // segment of this block
    const long long b = blockIdx.x;
    int si = 0;
    #pragma unroll 1
    while (si + 1 < p.nseg && b >= p.seg[si + 1].blk0) ++si;
    const Seg<T>& S = p.seg[si];
    const long long u = b - S.blk0;
    const int tileidx = (int)(u % S.tiles);
    const int unit = (int)(u / S.tiles);
    int ob, oe;
    if (MODE == M_POT) {
        ob = unit * S.opg;
        oe = min(S.norb, ob + S.opg);
    } else {
        ob = unit;
        oe = unit + 1;
    }

    const int LT = p.LT, n = S.n, N = S.N, hl = p.hl, rowlen = S.rowlen;
    const int a0 = tileidx * LT;
    const int lt = min(LT, N - a0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int spw = 32 / LT;
    const int line = lane & (LT - 1);
    const int slot = warp * spw + lane / LT;
    const int nslots = (NTHREADS / 32) * spw;
    const int nchunks = (n + R - 1) / R;
    const long long P = S.P;
    const bool line_ok = line < lt;
    const T* srow_line = tile + line * rowlen;

    constexpr int CPT = (MODE == M_POT) ? POT_OUT / R : 1;
    Acc<T> racc[CPT][R];   // M_POT: density per owned output, kept across orbitals

    #pragma unroll 1
    for (int orb = ob; orb < oe; ++orb) {
        // ---------------- stage the lines (with periodic halos) in smem
        #pragma unroll 1
        for (int r = warp; r < LT; r += NTHREADS / 32) {
            T* row = tile + r * rowlen + hl;
            if (r < lt) {
                const int a = a0 + r;
                if (MODE == M_UNCOMP) {
                    // line a = (x3, x2) of the interleaved coarse array; element
                    // x1 of it is c^mu[i3][i2][i1], mu = a1 + 2 a2 + 4 a3
                    const int x3 = a / S.N2, x2 = a - x3 * S.N2;
                    const int i3 = x3 >> 1, i2 = x2 >> 1;
                    const int mu23 = 2 * (x2 & 1) + 4 * (x3 & 1);
                    const long long m = P >> 3;
                    const T* cc = S.in + (long long)orb * P;
                    const T* cf = cc + m;
                    const long long cb = ((long long)i3 * S.n2 + i2) * S.n1;
                    #pragma unroll 2
                    for (int i = lane; i < n; i += 32) {
                        const int mu = mu23 + (i & 1);
                        const long long ci = cb + (i >> 1);
                        row[i] = (mu == 0) ? cc[ci] : cf[ci * 7 + mu - 1];
                    }
                } else {
                    const T* src = S.in + (long long)orb * P + (long long)a * n;
                    #pragma unroll 4
                    for (int i = lane; i < n; i += 32) row[i] = src[i];
                }
            } else {
                for (int i = lane; i < n; i += 32) row[i] = T(0);
            }
        }
        __syncthreads();
        #pragma unroll 1
        for (int r = warp; r < LT; r += NTHREADS / 32) {
            T* row = tile + r * rowlen;
            for (int j = lane; j < rowlen; j += 32) {
                if (j < hl || j >= hl + n) {
                    int x = (j - hl) % n;
                    if (x < 0) x += n;
                    row[j] = row[hl + x];
                }
            }
        }
        __syncthreads();

        // ---------------- convolve, epilogue
        Acc<T> e;   // energy partial of this orbital
        double occ = 0.0;
        if (MODE == M_POT) occ = S.occ ? S.occ[orb] : 1.0;
        const long long obase = (long long)orb * P;

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
                for (int r = 0; r < R; ++r) acc[r] = T(0);
                if (MODE == M_KMID || MODE == M_KLAST) {
                    if (S.in2 != nullptr && line_ok) {
                        const T* kp = S.in2 + obase + (long long)(a0 + line) * n + i0;
                        #pragma unroll
                        for (int r = 0; r < R; ++r)
                            if (i0 + r < n) acc[r] = kp[r];
                    }
                }
                conv_chunk<T, KIND, R>(srow_line + i0, p, acc);
                if (!line_ok) continue;
                #pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int I = i0 + r;
                    if (I >= n) continue;
                    const long long oidx = (long long)I * N + a0 + line;
                    if (MODE == M_PLAIN || MODE == M_UNCOMP) {
                        S.out[obase + oidx] = acc[r];
                    } else if (MODE == M_COMP) {
                        // output (X3 = I, a = X2 * N1 + X1) -> compressed position
                        const int a = a0 + line;
                        const int X2 = a / S.N1, X1 = a - X2 * S.N1;
                        const int mu = (X1 & 1) + 2 * (X2 & 1) + 4 * (I & 1);
                        const long long ci =
                            ((long long)(I >> 1) * S.n2 + (X2 >> 1)) * S.n1 + (X1 >> 1);
                        T* cc0 = S.out + obase;
                        if (mu == 0) cc0[ci] = acc[r];
                        else cc0[(P >> 3) + ci * 7 + mu - 1] = acc[r];
                    } else if (MODE == M_KMID) {
                        S.out[obase + oidx] = acc[r];
                        S.out2[obase + oidx] = srow_line[hl + I];
                    } else if (MODE == M_KLAST) {
                        if (S.out) S.out[obase + oidx] = acc[r];
                        const T k0 = S.aux ? S.aux[obase + oidx] : T(0);
                        e.fma_add(srow_line[hl + I], acc[r] - k0);
                    } else if (MODE == M_POT) {
                        const T psi = acc[r];
                        if (S.aux) {
                            const T y = S.aux[oidx] * psi;
                            if (S.out) S.out[obase + oidx] = y;
                            e.fma_add(y, psi);
                        }
                        if (S.rho) racc[cc][r].add((T)occ * psi * psi);
                    }
                }
            }
        }

        if ((MODE == M_POT && S.aux) || MODE == M_KLAST) {
            const double t = block_sum(e.get(), red);
            if (threadIdx.x == 0) S.part[(long long)orb * S.tiles + tileidx] = t;
        }
        __syncthreads();   // smem reused by the next orbital
    }

    if (MODE == M_POT && S.rho != nullptr && line_ok) {
        const int grp = unit;
        #pragma unroll
        for (int cc = 0; cc < CPT; ++cc) {
            const int c = slot + cc * nslots;
            if (c >= nchunks) continue;
            #pragma unroll
            for (int r = 0; r < R; ++r) {
                const int I = c * R + r;
                if (I >= n) continue;
                const long long oidx = (long long)I * N + a0 + line;
                if (S.rho_gstride == 0) S.rho[oidx] += racc[cc][r].get();
                else S.rho[grp * S.rho_gstride + oidx] = racc[cc][r].get();
            }
        }
    }
}

}  // namespace wvl
