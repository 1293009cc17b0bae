// Instantiations of the warp-specialised degridding kernels with the tiles of candidate 3 (the
// tensor-core gridding configuration), all exact supports.
#include "resample_ws.cuh"

namespace awg {
AWG_FOR_WS_A(AWG_INSTANTIATE_DEGRID_WS3)
AWG_FOR_WS_B(AWG_INSTANTIATE_DEGRID_WS3)
}  // namespace awg
