// Instantiations of the warp-specialised degridding kernels with the tiles of candidate 3 (the
// tensor-core configuration) for the supports whose windows are wider than one tensor-core tile.
#include "resample_ws.cuh"

namespace awg {
AWG_FOR_WS3(AWG_INSTANTIATE_DEGRID_WS3)
}  // namespace awg
