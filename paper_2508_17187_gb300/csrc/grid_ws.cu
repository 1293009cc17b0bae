// Instantiations of the warp-specialised gridding kernels, supports 8-32.
#include "resample_ws.cuh"

namespace awg {
AWG_FOR_WS_A(AWG_INSTANTIATE_GRID_WS)
}  // namespace awg
