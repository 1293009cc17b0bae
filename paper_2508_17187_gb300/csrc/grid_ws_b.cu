// Instantiations of the warp-specialised gridding kernels, supports 40-64.
#include "resample_ws.cuh"

namespace awg {
AWG_FOR_WS_B(AWG_INSTANTIATE_GRID_WS)
}  // namespace awg
