// Instantiations of the tensor-core gridding kernels, supports 40-64.
#include "resample_mma.cuh"

namespace awg {
AWG_FOR_WS_B(AWG_INSTANTIATE_GRID_MMA)
}  // namespace awg
