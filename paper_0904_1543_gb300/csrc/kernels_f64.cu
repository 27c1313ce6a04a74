// FP64 instantiations of the pass kernels.
#include "kernels_impl.cuh"

namespace wvl {
WVL_INSTANTIATE_LAUNCH(double)
}  // namespace wvl
