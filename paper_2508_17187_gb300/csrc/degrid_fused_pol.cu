// Instantiations of the fused degridding kernels with pol mixing (the base passes of full-polarisation
// CF sets: 4 pols, 2-4 outer-product terms, exact supports).
#include "resample_sep.cuh"

namespace awg {
AWG_FOR_FUSED_MIX(AWG_INSTANTIATE_DEGRID_FUSED_MIX, 2)
AWG_FOR_FUSED_MIX(AWG_INSTANTIATE_DEGRID_FUSED_MIX, 3)
AWG_FOR_FUSED_MIX(AWG_INSTANTIATE_DEGRID_FUSED_MIX, 4)
}  // namespace awg
