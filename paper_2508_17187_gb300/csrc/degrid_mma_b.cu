// Instantiations of the tensor-core degridding kernels, supports 40-56.
#include "resample_mma_dg.cuh"

namespace awg {
AWG_FOR_MMA_DG_B(AWG_INSTANTIATE_DEGRID_MMA)
}  // namespace awg
