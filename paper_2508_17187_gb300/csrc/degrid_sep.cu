// Instantiations of the separable-CF degridding kernel for every class and pol count.
#include "resample_sep.cuh"

namespace awg {
AWG_FOR_SEP_CLASSES_AND_POLS(AWG_INSTANTIATE_DEGRID_SEP)
}  // namespace awg
