// Instantiations of the tensor-core degridding kernels, supports 8-32.
#include "resample_mma_dg.cuh"

namespace awg {
AWG_FOR_MMA_DG_A(AWG_INSTANTIATE_DEGRID_MMA)
}  // namespace awg
