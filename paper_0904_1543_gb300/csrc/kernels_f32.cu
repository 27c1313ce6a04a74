// FP32 instantiations of the pass kernels (energies accumulate in FP64, the
// density in compensated pairs, then FP64).
#include "kernels_impl.cuh"

namespace wvl {
WVL_INSTANTIATE_LAUNCH(float)
}  // namespace wvl
