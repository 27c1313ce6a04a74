// FP32 instantiations of the pass kernels (reductions stay compensated/double).
#include "kernels_impl.cuh"

namespace wvl {
WVL_INSTANTIATE_LAUNCH(float)
}  // namespace wvl
