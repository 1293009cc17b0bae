// Instantiations of the gridding kernels with BF16 CF storage for every class and pol count.
#include "resample.cuh"

namespace awg {
AWG_FOR_CLASSES_AND_POLS(AWG_INSTANTIATE_GRID, true)
}  // namespace awg
