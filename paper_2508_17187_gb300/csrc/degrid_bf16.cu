// Instantiations of the degridding kernels with BF16 CF storage for every class and pol count.
#include "resample.cuh"

namespace awg {
AWG_FOR_CLASSES_AND_POLS(AWG_INSTANTIATE_DEGRID, true)
}  // namespace awg
