// Instantiations of the fused gridding kernels for CF sets of 3 outer-product terms, configuration 1.
#include "resample_sep.cuh"

namespace awg {
AWG_FOR_FUSED(AWG_INSTANTIATE_GRID_FUSED_C1, 3)
}  // namespace awg
