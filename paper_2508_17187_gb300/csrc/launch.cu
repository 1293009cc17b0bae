// Host launch code: per-class dispatch of the gridding / degridding kernels, zeroing of dropped
// samples after degridding, and the taper normalisation kernel (grid_normalize).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "resample_mma_dg.cuh"

namespace awg {

AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_GRID, false)
AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_GRID, true)
AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_DEGRID, false)
AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_DEGRID, true)
AWG_FOR_SEP_CLASSES_AND_POLS(AWG_DECLARE_GRID_SEP)
AWG_FOR_SEP_CLASSES_AND_POLS(AWG_DECLARE_DEGRID_SEP)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_GRID_EXACT, 0)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_DEGRID_EXACT, 0)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_GRID_EXACT, 1)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_DEGRID_EXACT, 1)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_GRID_EXACT, 2)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_DEGRID_EXACT, 2)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_GRID_EXACT, 3)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_DEGRID_EXACT, 3)
AWG_FOR_WS_A(AWG_DECLARE_GRID_MMA)
AWG_FOR_WS_B(AWG_DECLARE_GRID_MMA)
AWG_FOR_WS3(AWG_DECLARE_DEGRID_WS3)
AWG_FOR_MMA_DG_A(AWG_DECLARE_DEGRID_MMA)
AWG_FOR_MMA_DG_B(AWG_DECLARE_DEGRID_MMA)
AWG_FOR_WS_A(AWG_DECLARE_GRID_WS)
AWG_FOR_WS_B(AWG_DECLARE_GRID_WS)
AWG_FOR_WS_A(AWG_DECLARE_DEGRID_WS)
AWG_FOR_WS_B(AWG_DECLARE_DEGRID_WS)
AWG_FOR_FUSED(AWG_DECLARE_GRID_FUSED, 2)
AWG_FOR_FUSED(AWG_DECLARE_GRID_FUSED, 3)
AWG_FOR_FUSED(AWG_DECLARE_GRID_FUSED, 4)
AWG_FOR_FUSED(AWG_DECLARE_DEGRID_FUSED, 2)
AWG_FOR_FUSED(AWG_DECLARE_DEGRID_FUSED, 3)
AWG_FOR_FUSED(AWG_DECLARE_DEGRID_FUSED, 4)
AWG_FOR_FUSED(AWG_DECLARE_GRID_FUSED_C1, 2)
AWG_FOR_FUSED(AWG_DECLARE_GRID_FUSED_C1, 3)
AWG_FOR_FUSED(AWG_DECLARE_GRID_FUSED_C1, 4)
AWG_FOR_FUSED(AWG_DECLARE_DEGRID_FUSED_C1, 2)
AWG_FOR_FUSED(AWG_DECLARE_DEGRID_FUSED_C1, 3)
AWG_FOR_FUSED(AWG_DECLARE_DEGRID_FUSED_C1, 4)
AWG_FOR_FUSED_MIX(AWG_DECLARE_GRID_FUSED_MIX, 2)
AWG_FOR_FUSED_MIX(AWG_DECLARE_GRID_FUSED_MIX, 3)
AWG_FOR_FUSED_MIX(AWG_DECLARE_GRID_FUSED_MIX, 4)
AWG_FOR_FUSED_MIX(AWG_DECLARE_DEGRID_FUSED_MIX, 2)
AWG_FOR_FUSED_MIX(AWG_DECLARE_DEGRID_FUSED_MIX, 3)
AWG_FOR_FUSED_MIX(AWG_DECLARE_DEGRID_FUSED_MIX, 4)

namespace {

int sm_count(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return sms > 0 ? sms : 1;
}

bool class_present(const CfSetImpl* cf, int c) {
  for (int i = 0; i < cf->slots.n; ++i)
    if (class_of_support(cf->slots.S[i]) == c) return true;
  return false;
}

template <bool BF16>
awg_status grid_class(int c, int P, const GridArgs& a, int sms, cudaStream_t st) {
#define AWG_CASE(C, PP, BF)                                    \
  if (c == C && P == PP) return run_grid<C, PP, BF16>(a, sms, st);
  AWG_FOR_CLASSES_AND_POLS(AWG_CASE, BF16)
#undef AWG_CASE
  return set_error(AWG_ERR_UNSUPPORTED, "no gridding kernel for this class / pol count");
}

// The warp-specialised and tensor-core kernels take P-contiguous visibilities and grids (no
// Mueller element passes or pol mixing), 16-byte aligned buffers (the grid and its compensation
// grid take 16-byte atomics), and grids of at most 32768 pixels (window
// origins packed in 16 bits); other calls on candidate 2 run the cp.async kernels of its tiles.
bool ws_grid_ok(const GridArgs& a, int P) {
  return a.mix == nullptr && a.vstride == P && a.voff == 0 && a.gstride == P && a.goff == 0 && a.N <= 32768 &&
         ((uintptr_t)a.vis & 15) == 0 && ((uintptr_t)a.weight & 15) == 0 && ((uintptr_t)a.grid & 15) == 0 &&
         ((uintptr_t)a.grid_lo & 15) == 0;
}

bool ws_degrid_ok(const DegridArgs& a, int P) {
  return a.mix == nullptr && a.gstride == P && a.goff == 0 && a.N <= 32768 && ((uintptr_t)a.grid & 15) == 0;
}

// Separable kernels run once per distinct support (slot): the exact-support kernel when there is
// one for S, else the class kernel restricted to the slot's items.
awg_status grid_slot_sep(int S, int cand, int slot, int P, const GridArgs& a, int sms, cudaStream_t st) {
  if (has_exact(S)) {   // the plan binned this support by its exact-kernel tile
    if (cand == 2 && ws_grid_ok(a, P)) {
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_grid_ws<SS, PP>(a, slot, sms, st);
      AWG_FOR_WS_A(AWG_CASE)
      AWG_FOR_WS_B(AWG_CASE)
#undef AWG_CASE
    }
    if (cand == 3 && ws_grid_ok(a, P)) {
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_grid_mma<SS, PP>(a, slot, sms, st);
      AWG_FOR_WS_A(AWG_CASE)
      AWG_FOR_WS_B(AWG_CASE)
#undef AWG_CASE
    }
#define AWG_CASE(SS, PP, CC) \
  if (S == SS && P == PP && cand == CC) return run_grid_exact<SS, PP, CC>(a, slot, sms, st);
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 0)
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 1)
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 2)
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 3)
#undef AWG_CASE
    return set_error(AWG_ERR_UNSUPPORTED, "no exact-support kernel for this support / pol count");
  }
  const int c = class_of_support(S);
#define AWG_CASE(C, PP) \
  if (c == C && P == PP) return run_grid_sep<C, PP>(a, slot, sms, st);
  AWG_FOR_SEP_CLASSES_AND_POLS(AWG_CASE)
#undef AWG_CASE
  return set_error(AWG_ERR_UNSUPPORTED, "no separable gridding kernel for this support / pol count");
}

// Fused kernels: one record per sample of a CF set of rk outer-product terms (the pol-mixing
// instances when a.mix is set).
// cand: the support's configuration (0 or 1; the plan binned the support by its tile).
awg_status grid_slot_fused(int S, int rk, int cand, int slot, int P, const GridArgs& a, int sms, cudaStream_t st) {
  if (a.mix != nullptr) {
    if (cand != 0) return set_error(AWG_ERR_UNSUPPORTED, "pol-mixing kernels have one configuration");
#define AWG_CASE(SS, PP, RR) \
  if (S == SS && P == PP && rk == RR) return run_grid_fused<SS, PP, RR, true>(a, slot, sms, st);
    AWG_FOR_FUSED_MIX(AWG_CASE, 2)
    AWG_FOR_FUSED_MIX(AWG_CASE, 3)
    AWG_FOR_FUSED_MIX(AWG_CASE, 4)
#undef AWG_CASE
    return set_error(AWG_ERR_UNSUPPORTED, "no pol-mixing gridding kernel for this support / pol count / rank");
  }
  if (cand == 1) {
#define AWG_CASE(SS, PP, RR) \
  if (S == SS && P == PP && rk == RR) return run_grid_fused<SS, PP, RR, false, 1>(a, slot, sms, st);
    AWG_FOR_FUSED(AWG_CASE, 2)
    AWG_FOR_FUSED(AWG_CASE, 3)
    AWG_FOR_FUSED(AWG_CASE, 4)
#undef AWG_CASE
    return set_error(AWG_ERR_UNSUPPORTED, "no fused gridding kernel for this support / pol count / rank");
  }
#define AWG_CASE(SS, PP, RR) \
  if (S == SS && P == PP && rk == RR) return run_grid_fused<SS, PP, RR>(a, slot, sms, st);
  AWG_FOR_FUSED(AWG_CASE, 2)
  AWG_FOR_FUSED(AWG_CASE, 3)
  AWG_FOR_FUSED(AWG_CASE, 4)
#undef AWG_CASE
  return set_error(AWG_ERR_UNSUPPORTED, "no fused gridding kernel for this support / pol count / rank");
}

// cand: the support's configuration (0 or 1; the plan binned the support by its tile).
awg_status degrid_slot_fused(int S, int rk, int cand, int slot, int P, const DegridArgs& a, int sms, cudaStream_t st) {
  if (a.mix != nullptr) {
    if (cand != 0) return set_error(AWG_ERR_UNSUPPORTED, "pol-mixing kernels have one configuration");
#define AWG_CASE(SS, PP, RR) \
  if (S == SS && P == PP && rk == RR) return run_degrid_fused<SS, PP, RR, true>(a, slot, sms, st);
    AWG_FOR_FUSED_MIX(AWG_CASE, 2)
    AWG_FOR_FUSED_MIX(AWG_CASE, 3)
    AWG_FOR_FUSED_MIX(AWG_CASE, 4)
#undef AWG_CASE
    return set_error(AWG_ERR_UNSUPPORTED, "no pol-mixing degridding kernel for this support / pol count / rank");
  }
  if (cand == 1) {
#define AWG_CASE(SS, PP, RR) \
  if (S == SS && P == PP && rk == RR) return run_degrid_fused<SS, PP, RR, false, 1>(a, slot, sms, st);
    AWG_FOR_FUSED(AWG_CASE, 2)
    AWG_FOR_FUSED(AWG_CASE, 3)
    AWG_FOR_FUSED(AWG_CASE, 4)
#undef AWG_CASE
    return set_error(AWG_ERR_UNSUPPORTED, "no fused degridding kernel for this support / pol count / rank");
  }
#define AWG_CASE(SS, PP, RR) \
  if (S == SS && P == PP && rk == RR) return run_degrid_fused<SS, PP, RR>(a, slot, sms, st);
  AWG_FOR_FUSED(AWG_CASE, 2)
  AWG_FOR_FUSED(AWG_CASE, 3)
  AWG_FOR_FUSED(AWG_CASE, 4)
#undef AWG_CASE
  return set_error(AWG_ERR_UNSUPPORTED, "no fused degridding kernel for this support / pol count / rank");
}

awg_status degrid_slot_sep(int S, int cand, int slot, int P, const DegridArgs& a, int sms, cudaStream_t st) {
  if (has_exact(S)) {   // the plan binned this support by its exact-kernel tile
    if (cand == 2 && ws_degrid_ok(a, P)) {
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_degrid_ws<SS, PP>(a, slot, sms, st);
      AWG_FOR_WS_A(AWG_CASE)
      AWG_FOR_WS_B(AWG_CASE)
#undef AWG_CASE
    }
    if (cand == 3 && ws_degrid_ok(a, P)) {   // tensor cores where the window fits one tile row
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_degrid_mma<SS, PP>(a, slot, sms, st);
      AWG_FOR_MMA_DG_A(AWG_CASE)
      AWG_FOR_MMA_DG_B(AWG_CASE)
#undef AWG_CASE
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_degrid_ws<SS, PP, 3>(a, slot, sms, st);
      AWG_FOR_WS3(AWG_CASE)
#undef AWG_CASE
    }
#define AWG_CASE(SS, PP, CC) \
  if (S == SS && P == PP && cand == CC) return run_degrid_exact<SS, PP, CC>(a, slot, sms, st);
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 0)
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 1)
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 2)
    AWG_FOR_EXACT_AND_POLS(AWG_CASE, 3)
#undef AWG_CASE
    return set_error(AWG_ERR_UNSUPPORTED, "no exact-support kernel for this support / pol count");
  }
  const int c = class_of_support(S);
#define AWG_CASE(C, PP) \
  if (c == C && P == PP) return run_degrid_sep<C, PP>(a, slot, sms, st);
  AWG_FOR_SEP_CLASSES_AND_POLS(AWG_CASE)
#undef AWG_CASE
  return set_error(AWG_ERR_UNSUPPORTED, "no separable degridding kernel for this support / pol count");
}

template <bool BF16>
awg_status degrid_class(int c, int P, const DegridArgs& a, int sms, cudaStream_t st) {
#define AWG_CASE(C, PP, BF)                                    \
  if (c == C && P == PP) return run_degrid<C, PP, BF16>(a, sms, st);
  AWG_FOR_CLASSES_AND_POLS(AWG_CASE, BF16)
#undef AWG_CASE
  return set_error(AWG_ERR_UNSUPPORTED, "no degridding kernel for this class / pol count");
}

// Taper correction, one pixel (its P pols) per thread: rows are dealt to the blocks in turn and
// a block's threads stride the row's pixels, so the index math is 32-bit with no division; the P
// complex values of a pixel move as float4 accesses (VEC: P = 2, 4 on a 16-byte aligned image) or
// float2 accesses.
template <int P, bool VEC>
__global__ void k_normalize(float2* __restrict__ img, const float* __restrict__ inv_taper,
                            const double* __restrict__ sumwt, int N, int direction) {
  float sp[P];
#pragma unroll
  for (int p = 0; p < P; ++p) sp[p] = (direction == 0 && sumwt) ? (float)(1.0 / sumwt[p]) : 1.f;
  for (int y = blockIdx.x; y < N; y += gridDim.x) {
    const float ty = inv_taper[y];
    float2* row = img + (size_t)y * N * P;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
      const float s = inv_taper[x] * ty;
      if constexpr (!VEC) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          float2 v = row[(size_t)x * P + p];
          v.x *= s * sp[p];
          v.y *= s * sp[p];
          row[(size_t)x * P + p] = v;
        }
      } else {
        float4* px = reinterpret_cast<float4*>(row + (size_t)x * P);
#pragma unroll
        for (int q = 0; q < P / 2; ++q) {
          float4 v = px[q];
          const float s0 = s * sp[2 * q], s1 = s * sp[2 * q + 1];
          v.x *= s0;
          v.y *= s0;
          v.z *= s1;
          v.w *= s1;
          px[q] = v;
        }
      }
    }
  }
}

}  // namespace

__global__ void k_zero_dropped(const int32_t* __restrict__ drop, const unsigned long long* __restrict__ counters,
                               float* __restrict__ vis_out, int P) {
  const int64_t nd = (int64_t)counters[1];
  const int64_t total = nd * 2 * P;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t d = i / (2 * P);
    vis_out[(int64_t)drop[d] * 2 * P + (i - d * 2 * P)] = 0.f;
  }
}

// vis_out[s] = sum over the rank terms of sample s (the CF's outer-product terms); pol p of sample
// s lands at s ostride + ooff + p, added to (accumulate 1) or subtracted from (accumulate -1) what
// is there.
__global__ void k_sum_terms(const float2* __restrict__ part, float2* __restrict__ vis_out, int64_t n, int rank,
                            int P, int ostride, int ooff, int accumulate) {
  const int64_t total = n * P;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int64_t s = i / P;
    const int p = (int)(i - s * P);
    float2 acc = make_float2(0.f, 0.f);
    for (int k = 0; k < rank; ++k) {
      const float2 v = part[(s * rank + k) * P + p];
      acc.x += v.x;
      acc.y += v.y;
    }
    float2* o = vis_out + s * ostride + ooff + p;
    if (accumulate) {
      const float2 prev = *o;
      acc = accumulate > 0 ? make_float2(prev.x + acc.x, prev.y + acc.y) : make_float2(prev.x - acc.x, prev.y - acc.y);
    }
    *o = acc;
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry points (the library does not link the
// driver library itself).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)f;
  });
  return fn;
}

// The grid c64 [N][N][P] as a TMA tensor of FP32 values whose box is `rows` rows of a window U
// pixels wide: P >= 2 a 3-D tensor (2P values of a pixel, x, y) with box (2P, U, rows); P = 1 a
// 2-D tensor (2N values of a row, y) with box (2 UB, rows), UB even, so that a box row is a whole
// number of 16-byte units.  Out-of-grid parts of a box read as zero.
awg_status make_grid_tensor_map(CUtensorMap* map, const void* grid, int N, int P, int U, int UB, int rows) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return set_error(AWG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUresult r;
  if (P >= 2) {
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * P), (cuuint64_t)N, (cuuint64_t)N};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * P * 4), (cuuint64_t)N * 2 * P * 4};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * P), (cuuint32_t)U, (cuuint32_t)rows};
    const cuuint32_t es[3] = {1, 1, 1};
    r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(grid), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * N), (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)N * 2 * 4};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * UB), (cuuint32_t)rows};
    const cuuint32_t es[2] = {1, 1};
    r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(grid), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return set_error(AWG_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return AWG_OK;
}

// Test hook of awg_debug_ws_withhold: the next warp-specialised launch withholds a hand-over.
static std::atomic<int> g_ws_withhold{0};

static GridArgs grid_args(const CfSetImpl* cf, const PlanImpl* pl, const void* vis, const float* weight, void* grid,
                          void* grid_lo, double* sumwt, int flags, int P) {
  GridArgs a;
  a.cf_shift = 0;
  a.vstride = a.gstride = P;
  a.voff = a.goff = 0;
  a.rec = pl->d_rec;
  a.items = pl->d_items;
  a.class_range = cf->separable ? pl->d_slot_range : pl->d_class_range;
  a.queue = pl->d_queue;
  a.cf = cf->d_data;
  a.cf_off = cf->d_off;
  a.OS = cf->p.oversampling;
  a.N = cf->p.grid_n;
  a.C = pl->C;
  a.flags = flags;
  a.has_phase = pl->has_phase;
  a.dl = pl->dl;
  a.dm = pl->dm;
  a.dn = pl->dn;
  a.uvw = pl->d_uvw;
  a.freq = pl->d_freq;
  a.row_dlm = pl->d_row_dlm;
  a.phasor = pl->has_phase ? pl->d_phasor : nullptr;
  a.vis = (const float*)vis;
  a.weight = weight;
  a.grid = (float*)grid;
  a.grid_lo = (float*)grid_lo;
  a.sumwt = sumwt;
  a.sep = (const float*)cf->d_sep;
  a.sep_off = cf->d_sep_off;
  a.n_sep_off = (int)cf->sep_offsets.size();
  a.rank = pl->rank;
  a.mix = nullptr;
  a.pmask = (1 << P) - 1;
  a.err = pl->d_counters + 3;
  a.withhold = 0;
  return a;
}

static DegridArgs degrid_args(const CfSetImpl* cf, const PlanImpl* pl, const void* grid, void* vis_out, int P) {
  DegridArgs a;
  a.cf_shift = 0;
  a.vstride = a.gstride = P;
  a.voff = a.goff = 0;
  a.accumulate = 0;
  a.rec = pl->d_rec;
  a.items = pl->d_items;
  a.class_range = cf->separable ? pl->d_slot_range : pl->d_class_range;
  a.queue = pl->d_queue;
  a.cf = cf->d_data;
  a.cf_off = cf->d_off;
  a.OS = cf->p.oversampling;
  a.N = cf->p.grid_n;
  a.C = pl->C;
  a.has_phase = pl->has_phase;
  a.dl = pl->dl;
  a.dm = pl->dm;
  a.dn = pl->dn;
  a.uvw = pl->d_uvw;
  a.freq = pl->d_freq;
  a.row_dlm = pl->d_row_dlm;
  a.phasor = pl->has_phase ? pl->d_phasor : nullptr;
  a.grid = (const float*)grid;
  // with several terms per CF every record writes its own row of the per-term buffer, summed later
  a.vis_out = pl->rank > 1 ? (float*)pl->d_part : (float*)vis_out;
  if (pl->rank > 1) a.vstride = P;
  a.sep = (const float*)cf->d_sep;
  a.sep_off = cf->d_sep_off;
  a.n_sep_off = (int)cf->sep_offsets.size();
  a.rank = pl->rank;
  a.mix = nullptr;
  a.pmask = (1 << P) - 1;
  a.err = pl->d_counters + 3;
  a.withhold = 0;
  return a;
}

awg_status plan_make_side_streams(PlanImpl* pl) {
  for (int k = 0; k < PlanImpl::kSideStreams; ++k) {
    AWG_CUDA_TRY(cudaStreamCreateWithFlags(&pl->side[k], cudaStreamNonBlocking));
    AWG_CUDA_TRY(cudaEventCreateWithFlags(&pl->join_ev[k], cudaEventDisableTiming));
  }
  AWG_CUDA_TRY(cudaEventCreateWithFlags(&pl->fork_ev, cudaEventDisableTiming));
  return AWG_OK;
}

void plan_free_side_streams(PlanImpl* pl) {
  // work still queued on a side stream completes first (the caller's stream waits for it)
  for (int k = 0; k < PlanImpl::kSideStreams; ++k) {
    if (pl->side[k]) cudaStreamDestroy(pl->side[k]);
    if (pl->join_ev[k]) cudaEventDestroy(pl->join_ev[k]);
    pl->side[k] = nullptr;
    pl->join_ev[k] = nullptr;
  }
  if (pl->fork_ev) cudaEventDestroy(pl->fork_ev);
  pl->fork_ev = nullptr;
}

// The per-support launches of one operator, spread over the plan's side streams: fork() orders
// them after the work already queued on the caller's stream, next() gives the stream of the next
// launch (the two side streams in turn, so at most two supports are in flight), and the
// destructor (or join()) makes the caller's stream wait for all of them.  Two launches in flight
// together share no state but the grid, to which gridding adds with atomics and from which
// degridding only reads: each launch has its own work-queue head and writes its own samples.  In
// a plan without side streams every launch stays on the caller's stream.
class SlotStreams {
 public:
  SlotStreams(PlanImpl* pl, cudaStream_t st) : pl_(pl), st_(st) {}
  ~SlotStreams() { join(); }
  awg_status fork() {
    if (!pl_->fork_ev) return AWG_OK;
    AWG_CUDA_TRY(cudaEventRecord(pl_->fork_ev, st_));
    forked_ = true;   // from here on the side streams are joined back, even after an error
    for (int k = 0; k < PlanImpl::kSideStreams; ++k) AWG_CUDA_TRY(cudaStreamWaitEvent(pl_->side[k], pl_->fork_ev, 0));
    return AWG_OK;
  }
  cudaStream_t next() { return forked_ ? pl_->side[n_++ % PlanImpl::kSideStreams] : st_; }
  awg_status join() {
    if (!forked_) return AWG_OK;
    forked_ = false;
    for (int k = 0; k < PlanImpl::kSideStreams; ++k) {
      AWG_CUDA_TRY(cudaEventRecord(pl_->join_ev[k], pl_->side[k]));
      AWG_CUDA_TRY(cudaStreamWaitEvent(st_, pl_->join_ev[k], 0));
    }
    return AWG_OK;
  }

 private:
  PlanImpl* pl_;
  cudaStream_t st_;
  bool forked_ = false;
  int n_ = 0;
};

static awg_status check_version(const CfSetImpl* cf, const PlanImpl* pl) {
  if (pl->slots_version != cf->slots_version)
    return set_error(AWG_ERR_INVALID_ARG, "the CF set was retuned after this plan was made; create a new plan");
  return AWG_OK;
}

awg_status launch_grid(CfSetImpl* cf, PlanImpl* pl, const void* vis, const float* weight, int P, void* grid,
                       void* grid_lo, double* sumwt, int flags, cudaStream_t st) {
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  awg_status s = check_version(cf, pl);
  if (s != AWG_OK) return s;
  pl->last_stream = st;
  if (pl->n == 0) return AWG_OK;
  GridArgs a = grid_args(cf, pl, vis, weight, grid, grid_lo, sumwt, flags, P);
  a.withhold = g_ws_withhold.exchange(0);
  const int sms = sm_count(pl->device);
  const bool bf16 = cf->p.cf_dtype == AWG_CF_BF16;
  if (cf->n_mb > 1 && cf->mb_elements) {
    // full-polarisation set stored per element (p, q): one single-pol pass per element, grid pol q
    // += conj(CF_pq) w_p V_p; the diagonal elements add their weights to sumwt[q]
    if (P != 4) return set_error(AWG_ERR_INVALID_ARG, "a full-polarisation CF set needs 4 pols");
    for (int e = 0; e < cf->n_elem; ++e) {
      GridArgs ae = a;
      ae.cf_shift = (int64_t)e * cf->n_base * pl->rank;
      ae.vstride = ae.gstride = 4;
      ae.voff = cf->elem_p[e];
      ae.goff = cf->elem_q[e];
      ae.sumwt = cf->elem_p[e] == cf->elem_q[e] ? sumwt + cf->elem_q[e] : nullptr;
      AWG_CUDA_TRY(cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st));
      SlotStreams ss(pl, st);
      if ((s = ss.fork()) != AWG_OK) return s;
      for (int i = cf->slots.n - 1; i >= 0; --i) {
        s = grid_slot_sep(cf->slots.S[i], cf->cand[cf->slots.S[i]], i, 1, ae, sms, ss.next());
        if (s != AWG_OK) return s;
      }
      if ((s = ss.join()) != AWG_OK) return s;
    }
    return AWG_OK;
  }
  // A full-polarisation set with fused kernels runs one 4-pol pass per base CF block k: grid pol q
  // gets conj(B_k) sum_p conj(s_pq) w_p V_p over the pols p of block k (mixing matrix mix_g[k]);
  // the weights of those pols go to sumwt.
  const int n_pass = cf->n_mb;
  if (n_pass > 1 && P != 4) return set_error(AWG_ERR_INVALID_ARG, "a full-polarisation CF set needs 4 pols");
  for (int k = 0; k < n_pass; ++k) {
    GridArgs ak = a;
    if (n_pass > 1) {
      ak.cf_shift = (int64_t)k * cf->n_base * cf->rank;   // factor offsets stride: the set's terms
      ak.mix = cf->d_mix + 32 * k;
      ak.pmask = cf->mb_pmask[k];
    }
    AWG_CUDA_TRY(cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st));
    if (cf->separable) {
      SlotStreams ss(pl, st);
      if ((s = ss.fork()) != AWG_OK) return s;
      for (int i = cf->slots.n - 1; i >= 0; --i) {   // largest supports first
        const cudaStream_t si = ss.next();
        s = cf->fused ? grid_slot_fused(cf->slots.S[i], cf->fused, cf->cand[cf->slots.S[i]], i, P, ak, sms, si)
                      : grid_slot_sep(cf->slots.S[i], cf->cand[cf->slots.S[i]], i, P, ak, sms, si);
        if (s != AWG_OK) return s;
      }
      if ((s = ss.join()) != AWG_OK) return s;
      continue;
    }
    for (int c = kNumClasses - 1; c >= 0; --c) {   // largest supports first
      if (!class_present(cf, c)) continue;
      s = bf16 ? grid_class<true>(c, P, ak, sms, st) : grid_class<false>(c, P, ak, sms, st);
      if (s != AWG_OK) return s;
    }
  }
  return AWG_OK;
}

// Per-term values summed, then dropped samples zeroed (after the kernels of launch_degrid).
static awg_status degrid_finish(PlanImpl* pl, void* vis_out, int P, int sms, cudaStream_t st, bool subtract) {
  if (pl->rank > 1) {   // dropped samples' rows are stale here and are zeroed next
    k_sum_terms<<<sms * 8, 256, 0, st>>>(pl->d_part, (float2*)vis_out, pl->n, pl->rank, P, P, 0, subtract ? -1 : 0);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  if (subtract) return AWG_OK;   // dropped samples keep their input
  k_zero_dropped<<<sms * 4, 256, 0, st>>>(pl->d_drop, pl->d_counters, (float*)vis_out, P);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

awg_status launch_degrid(CfSetImpl* cf, PlanImpl* pl, const void* grid, void* vis_out, int P, cudaStream_t st,
                         bool subtract) {
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  awg_status s = check_version(cf, pl);
  if (s != AWG_OK) return s;
  pl->last_stream = st;
  if (pl->n == 0) return AWG_OK;
  DegridArgs a = degrid_args(cf, pl, grid, vis_out, P);
  a.withhold = g_ws_withhold.exchange(0);
  if (subtract && pl->rank == 1) a.accumulate = -1;   // rank > 1: the per-term sums subtract
  const int sms = sm_count(pl->device);
  const bool bf16 = cf->p.cf_dtype == AWG_CF_BF16;
  if (cf->n_mb > 1 && cf->mb_elements) {
    // full-polarisation set stored per element: vis pol p = sum over elements (p, q) of CF_pq
    // applied to grid pol q; dropped samples keep the zeros written first
    if (P != 4) return set_error(AWG_ERR_INVALID_ARG, "a full-polarisation CF set needs 4 pols");
    if (!subtract) AWG_CUDA_TRY(cudaMemsetAsync(vis_out, 0, sizeof(float2) * 4 * (size_t)pl->n, st));
    for (int e = 0; e < cf->n_elem; ++e) {
      DegridArgs ae = a;
      ae.cf_shift = (int64_t)e * cf->n_base * pl->rank;
      ae.gstride = 4;
      ae.goff = cf->elem_q[e];
      if (pl->rank > 1) {   // per-term rows, one pol each, summed into vis pol p below
        ae.vis_out = (float*)pl->d_part;
        ae.vstride = 1;
        ae.voff = 0;
        ae.accumulate = 0;
      } else {
        ae.vis_out = (float*)vis_out;
        ae.vstride = 4;
        ae.voff = cf->elem_p[e];
        ae.accumulate = subtract ? -1 : 1;
      }
      AWG_CUDA_TRY(cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st));
      SlotStreams ss(pl, st);
      if ((s = ss.fork()) != AWG_OK) return s;
      for (int i = cf->slots.n - 1; i >= 0; --i) {
        s = degrid_slot_sep(cf->slots.S[i], cf->cand[cf->slots.S[i]], i, 1, ae, sms, ss.next());
        if (s != AWG_OK) return s;
      }
      if ((s = ss.join()) != AWG_OK) return s;
      if (pl->rank > 1) {
        k_sum_terms<<<sms * 8, 256, 0, st>>>(pl->d_part, (float2*)vis_out, pl->n, pl->rank, 1, 4, cf->elem_p[e],
                                             subtract ? -1 : 1);
        AWG_CUDA_TRY(cudaGetLastError());
        count_launches(1);
      }
    }
    // rows of dropped samples were never written by the kernels, but the sums above added their
    // stale per-term rows: zero them again (with subtract they keep their input)
    if (subtract) return AWG_OK;
    k_zero_dropped<<<sms * 4, 256, 0, st>>>(pl->d_drop, pl->d_counters, (float*)vis_out, 4);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AWG_OK;
  }
  // A full-polarisation set with fused kernels runs one 4-pol pass per base CF block k, which
  // writes the output pols p of block k: V_p = sum_q s_pq (B_k applied to grid pol q) (mixing
  // matrix mix_d[k]); its plans hold one record per sample.
  const int n_pass = cf->n_mb;
  if (n_pass > 1 && P != 4) return set_error(AWG_ERR_INVALID_ARG, "a full-polarisation CF set needs 4 pols");
  for (int k = 0; k < n_pass; ++k) {
    DegridArgs ak = a;
    if (n_pass > 1) {
      ak.cf_shift = (int64_t)k * cf->n_base * cf->rank;   // factor offsets stride: the set's terms
      ak.mix = cf->d_mix + 32 * k + 16;
      ak.pmask = cf->mb_pmask[k];
    }
    AWG_CUDA_TRY(cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st));
    if (cf->separable) {
      SlotStreams ss(pl, st);
      if ((s = ss.fork()) != AWG_OK) return s;
      for (int i = cf->slots.n - 1; i >= 0; --i) {
        const cudaStream_t si = ss.next();
        s = cf->fused ? degrid_slot_fused(cf->slots.S[i], cf->fused, cf->cand[cf->slots.S[i]], i, P, ak, sms, si)
                      : degrid_slot_sep(cf->slots.S[i], cf->cand[cf->slots.S[i]], i, P, ak, sms, si);
        if (s != AWG_OK) return s;
      }
      if ((s = ss.join()) != AWG_OK) return s;
    } else {
      for (int c = kNumClasses - 1; c >= 0; --c) {
        if (!class_present(cf, c)) continue;
        s = bf16 ? degrid_class<true>(c, P, ak, sms, st) : degrid_class<false>(c, P, ak, sms, st);
        if (s != AWG_OK) return s;
      }
    }
  }
  return degrid_finish(pl, vis_out, P, sms, st, subtract);
}

__global__ void k_fill_ones(float* vis, float* weight, int64_t n_vis) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vis; i += stride) {
    vis[2 * i] = 1.f;
    vis[2 * i + 1] = 0.f;
    weight[i] = 1.f;
  }
}

awg_status autotune_supports(CfSetImpl* cf, const double* uvw, int64_t n_rows, const double* freq, int n_chan,
                             const int32_t* pa_bin, const int32_t* chan_sb, int P, cudaStream_t st, int32_t* choice,
                             float* ms_out) {
  for (int S = 0; S <= kMaxSupport; ++S) choice[S] = -1;
  if (ms_out)
    for (int i = 0; i < kNumCand * (kMaxSupport + 1); ++i) ms_out[i] = 0.f;
  // full tables and pol-mixing sets have one configuration; fused sets have two (0 and 1)
  if (!cf->separable || (cf->fused && cf->n_mb > 1)) return AWG_OK;
  const int n_cand = cf->fused ? 2 : kNumCand;
  const int N = cf->p.grid_n;
  const int64_t n = n_rows * (int64_t)n_chan;
  // unit visibilities and weights (a value-independent timing; zeros would skip the flushes)
  float *vis = nullptr, *wt = nullptr, *grid = nullptr, *out = nullptr;
  double* sumwt = nullptr;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = dev_alloc(p, bytes); };
  A((void**)&vis, sizeof(float2) * std::max<int64_t>(n * P, 1));
  A((void**)&wt, sizeof(float) * std::max<int64_t>(n * P, 1));
  A((void**)&out, sizeof(float2) * std::max<int64_t>(n * P, 1));
  A((void**)&grid, sizeof(float2) * (size_t)N * N * P);
  A((void**)&sumwt, sizeof(double) * P);
  cudaEvent_t ev[4] = {};
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  auto cleanup = [&]() {
    dev_free(vis); dev_free(wt); dev_free(out); dev_free(grid); dev_free(sumwt);
    for (auto& x : ev)
      if (x) cudaEventDestroy(x);
  };
  if (e != cudaSuccess) {
    cleanup();
    return cuda_error(e, "autotune allocation");
  }
  const int sms = sm_count(cf->device);
  awg_status s = AWG_OK;
  float best[kMaxSupport + 1];
  for (int S = 0; S <= kMaxSupport; ++S) best[S] = 3.4e38f;
  int8_t pick[kMaxSupport + 1] = {};
  for (int c = 0; c < n_cand && s == AWG_OK; ++c) {
    for (int S = 1; S <= kMaxSupport; ++S)
      if (has_exact(S)) cf->cand[S] = (int8_t)c;
    fill_slots(cf);
    awg_plan h = nullptr;
    s = plan_create((awg_cf_set)cf, uvw, n_rows, freq, n_chan, pa_bin, chan_sb, nullptr, st, &h);
    if (s != AWG_OK) break;
    PlanImpl* pl = (PlanImpl*)h;
    if (n > 0) {
      k_fill_ones<<<sms * 4, 256, 0, st>>>(vis, wt, n * P);
      count_launches(1);
      if ((e = cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)N * N * P, st)) != cudaSuccess ||
          (e = cudaMemsetAsync(sumwt, 0, sizeof(double) * P, st)) != cudaSuccess) {
        s = cuda_error(e, "autotune memset");
      }
      // warm-up pass over every support, then three timed passes of each support's launches
      if (s == AWG_OK) s = launch_grid(cf, pl, vis, wt, P, grid, nullptr, sumwt, 0, st);
      if (s == AWG_OK) s = launch_degrid(cf, pl, grid, out, P, st);
      const GridArgs ga = grid_args(cf, pl, vis, wt, grid, nullptr, sumwt, 0, P);
      const DegridArgs da = degrid_args(cf, pl, grid, out, P);
      for (int i = 0; i < cf->slots.n && s == AWG_OK; ++i) {
        const int S = cf->slots.S[i];
        if (!has_exact(S)) continue;
        float t = 3.4e38f;
        for (int rep = 0; rep < 3 && s == AWG_OK; ++rep) {
          if ((e = cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st)) != cudaSuccess) {
            s = cuda_error(e, "autotune memset");
            break;
          }
          cudaEventRecord(ev[0], st);
          s = cf->fused ? grid_slot_fused(S, cf->fused, c, i, P, ga, sms, st) : grid_slot_sep(S, c, i, P, ga, sms, st);
          cudaEventRecord(ev[1], st);
          if (s != AWG_OK) break;
          if ((e = cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st)) != cudaSuccess) {
            s = cuda_error(e, "autotune memset");
            break;
          }
          cudaEventRecord(ev[2], st);
          s = cf->fused ? degrid_slot_fused(S, cf->fused, c, i, P, da, sms, st)
                        : degrid_slot_sep(S, c, i, P, da, sms, st);
          cudaEventRecord(ev[3], st);
          if (s != AWG_OK) break;
          if ((e = cudaEventSynchronize(ev[3])) != cudaSuccess) {
            s = cuda_error(e, "autotune timing");
            break;
          }
          float tg = 0.f, td = 0.f;
          cudaEventElapsedTime(&tg, ev[0], ev[1]);
          cudaEventElapsedTime(&td, ev[2], ev[3]);
          t = std::min(t, tg + td);
        }
        if (ms_out) ms_out[c * (kMaxSupport + 1) + S] = t;
        if (t < best[S]) {
          best[S] = t;
          pick[S] = (int8_t)c;
        }
      }
    }
    if (s == AWG_OK) {
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_error(e, "autotune");
    }
    plan_destroy(h);
  }
  // the fastest candidate of every timed support (candidate 0 where nothing was timed)
  for (int S = 1; S <= kMaxSupport; ++S)
    if (has_exact(S)) {
      cf->cand[S] = s == AWG_OK ? pick[S] : 0;
      if (s == AWG_OK && best[S] < 3.4e38f) choice[S] = pick[S];
    }
  fill_slots(cf);
  cleanup();
  return s;
}

awg_status launch_normalize(CfSetImpl* cf, void* image, int P, const double* sumwt, int direction, cudaStream_t st) {
  if (cudaSetDevice(cf->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  const int sms = sm_count(cf->device);
  const int N = cf->p.grid_n;
  const int blocks = std::min(N, sms * 16);
  const int threads = std::min(256, (N + 31) / 32 * 32);
  float2* img = (float2*)image;
  const bool vec = ((uintptr_t)image & 15) == 0;
  if (P == 1) k_normalize<1, false><<<blocks, threads, 0, st>>>(img, cf->d_inv_taper, sumwt, N, direction);
  else if (P == 2 && vec) k_normalize<2, true><<<blocks, threads, 0, st>>>(img, cf->d_inv_taper, sumwt, N, direction);
  else if (P == 2) k_normalize<2, false><<<blocks, threads, 0, st>>>(img, cf->d_inv_taper, sumwt, N, direction);
  else if (vec) k_normalize<4, true><<<blocks, threads, 0, st>>>(img, cf->d_inv_taper, sumwt, N, direction);
  else k_normalize<4, false><<<blocks, threads, 0, st>>>(img, cf->d_inv_taper, sumwt, N, direction);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

}  // namespace awg

extern "C" awg_status awg_debug_ws_withhold(int32_t on) {
  if (on != 0 && on != 1) return awg::set_error(AWG_ERR_INVALID_ARG, "on must be 0 or 1");
  awg::g_ws_withhold.store(on);
  return AWG_OK;
}
