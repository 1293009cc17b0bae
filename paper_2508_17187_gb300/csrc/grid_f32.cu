// Instantiations of the gridding kernels with FP32 CF storage for every class and pol count.
#include "resample.cuh"

namespace awg {
AWG_FOR_CLASSES_AND_POLS(AWG_INSTANTIATE_GRID, false)
}  // namespace awg
