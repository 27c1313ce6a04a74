// Tap geometry of the 1D filters shared by the pass and fused kernels, and
// the tap pairs of their packed FP32 form.  Host and device code (no device
// intrinsics), so the pairing can be checked on the CPU.
#pragma once
#include <cuda_runtime.h>

#include "wvl_internal.h"

namespace wvl {

// taps, parity offsets, extra window word, left halo (kind_geom on the host
// gives the same halos; the magic filter's follows from k0 = -7), and the
// taps skipped at each end (SKIP): the kinetic filter's a_{+-14} = -6.9e-18
// is 1/160 of the FP64 rounding error of the sum it enters (2^-53 sum |a_l|
// max|s| = 1.1e-15 max|s|), so the FP64 and FP32 kernels apply the 27 taps
// l = -13..13 (the window keeps its 29-tap geometry)
template <int KIND> struct KT;
template <> struct KT<K_MF>  { static constexpr int NT = 16, OFF0 = 0, OFF1 = 0, EXTRA = 0, HL = 8, SKIP = 0; };
template <> struct KT<K_MFT> { static constexpr int NT = 16, OFF0 = 0, OFF1 = 0, EXTRA = 0, HL = 7, SKIP = 0; };
template <> struct KT<K_KIN> { static constexpr int NT = 29, OFF0 = 0, OFF1 = 0, EXTRA = 0, HL = 14, SKIP = 1; };
template <> struct KT<K_SYN> { static constexpr int NT = 16, OFF0 = 0, OFF1 = 1, EXTRA = 1, HL = 8, SKIP = 0; };
template <> struct KT<K_ANA> { static constexpr int NT = 16, OFF0 = 1, OFF1 = 0, EXTRA = 1, HL = 8, SKIP = 0; };

// the taps of a filter that apply (the kinetic a_{+-14} do not)
template <int KIND>
__host__ __device__ constexpr bool tap_on(int t) {
    return t >= KT<KIND>::SKIP && t < KT<KIND>::NT - KT<KIND>::SKIP;
}

// Tap pairs of the packed FP32 convolutions: input (window element) j feeds
// outputs 2m and 2m + 1 of a chunk with taps t0 = d - off0 (even filter) and
// t1 = d - 1 - off1 (odd filter), d = j - 2m; a tap that does not apply is 0.
// One fma.rn.f32x2 then updates both outputs (two FMAs per lane per
// instruction), in the same order of taps as the scalar form.
template <int KIND>
void tap_pairs(const float (&f)[2][32], float2 (&tp)[32]) {
    for (int d = 0; d < 32; ++d) {
        const int t0 = d - KT<KIND>::OFF0, t1 = d - 1 - KT<KIND>::OFF1;
        tp[d].x = tap_on<KIND>(t0) ? f[0][t0] : 0.f;
        tp[d].y = tap_on<KIND>(t1) ? f[1][t1] : 0.f;
    }
}
template <int KIND>
__host__ __device__ constexpr bool pair_on(int d) {
    return d >= 0 && d < 32 &&
           (tap_on<KIND>(d - KT<KIND>::OFF0) || tap_on<KIND>(d - 1 - KT<KIND>::OFF1));
}

}  // namespace wvl
