// Hogbom CLEAN minor cycle on the GPU (the deconvolution step of the imaging major cycle,
// Sec. 5.2): repeatedly find the largest |residual| inside a search window, add gain * peak to
// the model at that pixel and subtract gain * peak * PSF centred there from the residual.
// Each iteration is three stream-ordered launches that read the peak from device memory, so the
// whole minor cycle needs no host round trip and can be captured in a CUDA graph.  The peak
// search and the update use separately rounded FP32 operations (no fused multiply-add), so the
// iteration sequence is reproducible by any IEEE FP32 implementation of the same steps.
#include <cuda_runtime.h>

#include "awg_internal.h"

namespace awg {
namespace {

constexpr int kCleanBlocks = 1024;
constexpr int kCleanThreads = 256;

struct CleanState {
  int active;    // 1 until the peak falls below the threshold
  int idx;       // pixel of the last component (y N + x)
  float gp;      // gain * peak of the last component (0 once inactive)
  int n_done;    // components found
};

struct BestPix {
  float a;   // |value|
  int i;     // linear pixel index
};

__device__ __forceinline__ BestPix better(BestPix p, BestPix q) {
  // larger |value| wins; equal values go to the lower index
  return (q.a > p.a || (q.a == p.a && q.i < p.i)) ? q : p;
}

__device__ BestPix block_best(BestPix b) {
  __shared__ float sa[32];
  __shared__ int si[32];
  for (int o = 16; o > 0; o >>= 1) {
    BestPix q;
    q.a = __shfl_xor_sync(0xffffffffu, b.a, o);
    q.i = __shfl_xor_sync(0xffffffffu, b.i, o);
    b = better(b, q);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = b.a;
    si[wid] = b.i;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    b.a = lane < nw ? sa[lane] : -1.f;
    b.i = lane < nw ? si[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      BestPix q;
      q.a = __shfl_xor_sync(0xffffffffu, b.a, o);
      q.i = __shfl_xor_sync(0xffffffffu, b.i, o);
      b = better(b, q);
    }
  }
  return b;   // valid in thread 0
}

// Largest |residual| of the window per block: block b takes window rows y0 + b, y0 + b + gridDim.x,
// ...; its threads stride the columns (coalesced, no division per pixel), 4 at a time with float4
// loads when the window's columns and the row pitch are multiples of 4 (VEC).
template <bool VEC>
__global__ void __launch_bounds__(kCleanThreads) k_absmax_partial(const float* __restrict__ res, int N, int x0, int x1,
                                                                   int y0, int y1, BestPix* __restrict__ part) {
  BestPix b{-1.f, 0x7fffffff};
  for (int y = y0 + blockIdx.x; y < y1; y += gridDim.x) {
    const float* row = res + (size_t)y * N;
    if constexpr (VEC) {
#pragma unroll 2
      for (int x = x0 + 4 * threadIdx.x; x < x1; x += 4 * blockDim.x) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(row + x));
        const int i = y * N + x;
        b = better(b, BestPix{fabsf(v.x), i});
        b = better(b, BestPix{fabsf(v.y), i + 1});
        b = better(b, BestPix{fabsf(v.z), i + 2});
        b = better(b, BestPix{fabsf(v.w), i + 3});
      }
    } else {
#pragma unroll 4
      for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) b = better(b, BestPix{fabsf(__ldg(row + x)), y * N + x});
    }
  }
  b = block_best(b);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void __launch_bounds__(1024) k_absmax_final(const BestPix* __restrict__ part, int n_part,
                                                       const float* __restrict__ res, float* __restrict__ model,
                                                       float gain, float threshold, CleanState* st) {
  BestPix b{-1.f, 0x7fffffff};
  for (int k = threadIdx.x; k < n_part; k += blockDim.x) b = better(b, part[k]);
  b = block_best(b);
  if (threadIdx.x == 0) {
    if (st->active && b.a >= 0.f && b.a >= threshold) {
      const float peak = res[b.i];
      const float gp = __fmul_rn(gain, peak);
      model[b.i] = __fadd_rn(model[b.i], gp);
      st->idx = b.i;
      st->gp = gp;
      st->n_done += 1;
    } else {
      st->active = 0;
      st->gp = 0.f;
    }
  }
}

// residual[y][x] -= g peak psf[y - py + Np/2][x - px + Np/2] where that PSF pixel exists: each
// thread takes 4 consecutive columns of rows blockIdx.y, blockIdx.y + gridDim.y, ... (one float4 of
// the residual when N is a multiple of 4), each product rounded before the subtraction.
template <bool VEC>
__global__ void __launch_bounds__(256) k_subtract_psf(float* __restrict__ res, const float* __restrict__ psf, int N,
                                                      int Np, const CleanState* __restrict__ st) {
  const float gp = st->gp;
  if (gp == 0.f) return;
  const int py = st->idx / N, px = st->idx - (st->idx / N) * N;
  const int xs = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (xs >= N) return;
  const int dx0 = xs - px + Np / 2;
  for (int y = blockIdx.y; y < N; y += gridDim.y) {
    const int dy = y - py + Np / 2;
    if (dy < 0 || dy >= Np) continue;
    float* r = res + (size_t)y * N + xs;
    const float* q = psf + (size_t)dy * Np;
    if constexpr (VEC) {
      float4 v = *reinterpret_cast<float4*>(r);
      float* e = &v.x;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int dx = dx0 + i;
        if (dx >= 0 && dx < Np) e[i] = __fsub_rn(e[i], __fmul_rn(gp, __ldg(q + dx)));
      }
      *reinterpret_cast<float4*>(r) = v;
    } else {
      for (int i = 0; i < 4 && xs + i < N; ++i) {
        const int dx = dx0 + i;
        if (dx >= 0 && dx < Np) r[i] = __fsub_rn(r[i], __fmul_rn(gp, __ldg(q + dx)));
      }
    }
  }
}

__global__ void k_clean_init(CleanState* st) {
  st->active = 1;
  st->idx = 0;
  st->gp = 0.f;
  st->n_done = 0;
}

}  // namespace
}  // namespace awg

using namespace awg;

extern "C" int64_t clean_hogbom_workspace_bytes(void) {
  return (int64_t)(sizeof(CleanState) + 16 + sizeof(BestPix) * kCleanBlocks);
}

extern "C" awg_status clean_hogbom(float* residual, float* model, int32_t N, const float* psf, int32_t psf_n,
                                   int32_t n_iter, float gain, float threshold, const int32_t* window, void* workspace,
                                   void* stream) {
  NvtxRange nvtx_range("awg clean_hogbom");
  if (!residual || !model || !psf || !workspace)
    return set_error(AWG_ERR_INVALID_ARG, "residual, model, psf and workspace must not be NULL");
  if (N < 1 || psf_n < 1 || n_iter < 0) return set_error(AWG_ERR_INVALID_ARG, "N, psf_n >= 1 and n_iter >= 0 required");
  if ((int64_t)N * N > ((int64_t)1 << 31) - 1) return set_error(AWG_ERR_UNSUPPORTED, "image too large");
  if (!(gain > 0.f && gain <= 1.f)) return set_error(AWG_ERR_INVALID_ARG, "gain must be in (0, 1]");
  if (!(threshold >= 0.f)) return set_error(AWG_ERR_INVALID_ARG, "threshold must be >= 0");
  int x0 = 0, x1 = N, y0 = 0, y1 = N;
  if (window) {
    x0 = window[0];
    x1 = window[1];
    y0 = window[2];
    y1 = window[3];
    if (x0 < 0 || y0 < 0 || x1 > N || y1 > N || x0 >= x1 || y0 >= y1)
      return set_error(AWG_ERR_INVALID_ARG, "window must satisfy 0 <= x0 < x1 <= N and 0 <= y0 < y1 <= N");
  }
  if (((uintptr_t)workspace & 15) != 0) return set_error(AWG_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  CleanState* st = (CleanState*)workspace;
  BestPix* part = (BestPix*)((char*)workspace + 16 + sizeof(CleanState));
  cudaStream_t s = (cudaStream_t)stream;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nb = std::min(kCleanBlocks, y1 - y0);   // peak search: window rows over up to kCleanBlocks blocks
  const bool vec4_search = N % 4 == 0 && x0 % 4 == 0 && (x1 - x0) % 4 == 0 && ((uintptr_t)residual & 15) == 0;
  // subtraction: 4 columns per thread, 256 threads per block in x, rows over about 8 blocks per SM
  const bool vec = N % 4 == 0 && ((uintptr_t)residual & 15) == 0;
  const int gx = (N + 4 * 256 - 1) / (4 * 256);
  const dim3 sub_grid(gx, (unsigned)std::max(1, std::min(N, std::max(sms, 1) * 8 / gx)));
  k_clean_init<<<1, 1, 0, s>>>(st);
  AWG_CUDA_TRY(cudaGetLastError());
  for (int it = 0; it < n_iter; ++it) {
    if (vec4_search) k_absmax_partial<true><<<nb, kCleanThreads, 0, s>>>(residual, N, x0, x1, y0, y1, part);
    else k_absmax_partial<false><<<nb, kCleanThreads, 0, s>>>(residual, N, x0, x1, y0, y1, part);
    k_absmax_final<<<1, 1024, 0, s>>>(part, nb, residual, model, gain, threshold, st);
    if (vec) k_subtract_psf<true><<<sub_grid, 256, 0, s>>>(residual, psf, N, psf_n, st);
    else k_subtract_psf<false><<<sub_grid, 256, 0, s>>>(residual, psf, N, psf_n, st);
  }
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1 + 3 * n_iter);
  return AWG_OK;
}

extern "C" awg_status clean_hogbom_components(const void* workspace, int32_t* n_done) {
  if (!workspace || !n_done) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CleanState h;
  AWG_CUDA_TRY(cudaMemcpy(&h, workspace, sizeof(CleanState), cudaMemcpyDeviceToHost));
  *n_done = h.n_done;
  return AWG_OK;
}
