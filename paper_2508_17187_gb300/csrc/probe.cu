// awg_fp32_fma_probe: the FP32 FMA rate of this GPU, the denominator of the gridding and
// degridding rooflines (both kernels are bound by the non-tensor FP32 pipe).
// awg_fp64_fma_probe: the FP64 FMA rate, the ceiling of the plain FP64 baseline kernels.
#include <cuda_runtime.h>

#include "awg_internal.h"

namespace awg {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (covers the FMA latency)

__global__ void __launch_bounds__(256) k_fma_probe(float* out, int64_t iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_fma_probe64(double* out, int64_t iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace awg

using namespace awg;

extern "C" awg_status awg_fp32_fma_probe(float* out, int32_t n_blocks, int64_t iters, void* stream, double* flop) {
  if (!out || !flop) return set_error(AWG_ERR_INVALID_ARG, "out and flop must not be NULL");
  if (n_blocks < 1 || iters < 1) return set_error(AWG_ERR_INVALID_ARG, "n_blocks and iters must be >= 1");
  // a and b keep x bounded (|x| stays below 1) and are not compile-time constants
  k_fma_probe<<<n_blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-4f);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  *flop = 2.0 * kChains * (double)iters * (double)n_blocks * 256.0;
  return AWG_OK;
}

extern "C" awg_status awg_fp64_fma_probe(double* out, int32_t n_blocks, int64_t iters, void* stream, double* flop) {
  if (!out || !flop) return set_error(AWG_ERR_INVALID_ARG, "out and flop must not be NULL");
  if (n_blocks < 1 || iters < 1) return set_error(AWG_ERR_INVALID_ARG, "n_blocks and iters must be >= 1");
  k_fma_probe64<<<n_blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999, 1e-4);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  *flop = 2.0 * kChains * (double)iters * (double)n_blocks * 256.0;
  return AWG_OK;
}
