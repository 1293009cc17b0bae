// Instantiations of the warp-specialised degridding kernels, supports 8-32.
#include "resample_ws.cuh"

namespace awg {
AWG_FOR_WS_A(AWG_INSTANTIATE_DEGRID_WS)
}  // namespace awg
