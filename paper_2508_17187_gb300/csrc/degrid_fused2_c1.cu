// Instantiations of the fused degridding kernels for CF sets of 2 outer-product terms, configuration 1.
#include "resample_sep.cuh"

namespace awg {
AWG_FOR_FUSED(AWG_INSTANTIATE_DEGRID_FUSED_C1, 2)
}  // namespace awg
