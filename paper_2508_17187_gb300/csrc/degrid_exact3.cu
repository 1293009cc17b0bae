// Instantiations of the exact-support separable degridding kernels (S = 8, 16, ..., 64), candidate 3
// (the tiles of the tensor-core configuration, for the calls the warp-specialised kernel cannot take).
#include "resample_sep.cuh"

namespace awg {
AWG_FOR_EXACT_AND_POLS(AWG_INSTANTIATE_DEGRID_EXACT, 3)
}  // namespace awg
