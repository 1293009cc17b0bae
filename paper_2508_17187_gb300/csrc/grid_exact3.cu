// Instantiations of the exact-support separable gridding kernels (S = 8, 16, ..., 64), candidate 3
// (the tiles of the tensor-core kernels, for the calls those cannot take).
#include "resample_sep.cuh"

namespace awg {
AWG_FOR_EXACT_AND_POLS(AWG_INSTANTIATE_GRID_EXACT, 3)
}  // namespace awg
