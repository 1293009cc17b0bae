// Instantiations of the tensor-core gridding kernels, supports 8-32.
#include "resample_mma.cuh"

namespace awg {
AWG_FOR_WS_A(AWG_INSTANTIATE_GRID_MMA)
}  // namespace awg
