// Double-FP32 ("double-float") arithmetic for the fused chain's FP64-grade
// form on the FP32 pipe (WVL_F64_DF).  A value is the unevaluated sum
// hi + lo of two binary32 numbers with |lo| <= ulp(hi) / 2 after
// normalisation: 48 significant bits, about 3.6e-15 relative.  The methods
// are the classical error-free transformations: Knuth's two-sum for
// additions and the FMA two-product (the rounding error of a * b is
// fma(a, b, -a b) exactly) for multiplications; the lo * lo term of a
// product (2^-48 relative) is dropped.
//
// Generic helpers (zero, mac, add, mul, Acc) let the fused kernels run on
// float, double and df alike.
#pragma once
#include <cuda_runtime.h>

namespace wvl {

struct df {
    float hi, lo;
};

__host__ __device__ inline df df_from(double d) {
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}
__host__ __device__ inline double df_to(df a) { return (double)a.hi + (double)a.lo; }

// |l| <= ulp(h) / 2 again (fast two-sum; valid as |s| >= |e|)
__device__ __forceinline__ df df_norm(float s, float e) {
    const float h = s + e;
    return {h, e - (h - s)};
}

// acc + f x: f.hi x.hi split exactly by the FMA two-product, the cross
// terms rounded, the addition by two-sum; left unnormalised (the lo parts
// of a filter's taps stay far below hi over the <= 29 terms of a window)
__device__ __forceinline__ df df_mac(df f, df x, df acc) {
    const float p = f.hi * x.hi;
    float e = fmaf(f.hi, x.hi, -p);
    e = fmaf(f.hi, x.lo, e);
    e = fmaf(f.lo, x.hi, e);
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (p - bb);
    return {s, acc.lo + (e + err)};
}

__device__ __forceinline__ df df_add(df a, df b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    return df_norm(s, (a.lo + b.lo) + err);
}

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_norm(p, e);
}

// ------------------------------------------------------------ generic ops
template <typename T> __device__ __forceinline__ T zero() { return T(0); }
template <> __device__ __forceinline__ df zero<df>() { return {0.f, 0.f}; }

__device__ __forceinline__ float mac(float f, float x, float a) { return fmaf(f, x, a); }
__device__ __forceinline__ double mac(double f, double x, double a) { return fma(f, x, a); }
__device__ __forceinline__ df mac(df f, df x, df a) { return df_mac(f, x, a); }

__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ df add(df a, df b) { return df_add(a, b); }

__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ df mul(df a, df b) { return df_mul(a, b); }

// normalised form of a stored result
__device__ __forceinline__ float settle(float a) { return a; }
__device__ __forceinline__ double settle(double a) { return a; }
__device__ __forceinline__ df settle(df a) { return df_norm(a.hi, a.lo); }

// from a double (the occupation, FP64 inputs) to the working type
template <typename T> __device__ __forceinline__ T from_double(double d) { return (T)d; }
template <> __device__ __forceinline__ df from_double<df>(double d) { return df_from(d); }

}  // namespace wvl
