// Host launch code: per-class dispatch of the gridding / degridding kernels, zeroing of dropped
// samples after degridding, and the taper normalisation kernel (grid_normalize).
#include <cuda_runtime.h>

#include "resample_sep.cuh"

namespace awg {

AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_GRID, false)
AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_GRID, true)
AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_DEGRID, false)
AWG_FOR_CLASSES_AND_POLS(AWG_DECLARE_DEGRID, true)
AWG_FOR_SEP_CLASSES_AND_POLS(AWG_DECLARE_GRID_SEP)
AWG_FOR_SEP_CLASSES_AND_POLS(AWG_DECLARE_DEGRID_SEP)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_GRID_EXACT)
AWG_FOR_EXACT_AND_POLS(AWG_DECLARE_DEGRID_EXACT)

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

// Separable kernels run once per distinct support (slot): the exact-support kernel when there is
// one for S, else the class kernel restricted to the slot's items.
awg_status grid_slot_sep(int S, int slot, int P, const GridArgs& a, int sms, cudaStream_t st) {
  if (has_exact(S)) {   // the plan binned this support by its exact-kernel tile
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_grid_exact<SS, PP>(a, slot, sms, st);
    AWG_FOR_EXACT_AND_POLS(AWG_CASE)
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

awg_status degrid_slot_sep(int S, int slot, int P, const DegridArgs& a, int sms, cudaStream_t st) {
  if (has_exact(S)) {   // the plan binned this support by its exact-kernel tile
#define AWG_CASE(SS, PP) \
  if (S == SS && P == PP) return run_degrid_exact<SS, PP>(a, slot, sms, st);
    AWG_FOR_EXACT_AND_POLS(AWG_CASE)
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

__global__ void k_normalize(float2* __restrict__ img, const float* __restrict__ inv_taper,
                            const double* __restrict__ sumwt, int N, int P, int direction) {
  const int64_t total = (int64_t)N * N * P;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int p = (int)(i % P);
    const int64_t pix = i / P;
    const int x = (int)(pix % N), y = (int)(pix / N);
    float s = inv_taper[x] * inv_taper[y];
    if (direction == 0 && sumwt) s *= (float)(1.0 / sumwt[p]);
    float2 v = img[i];
    v.x *= s;
    v.y *= s;
    img[i] = v;
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

// vis_out[s] = sum over the rank terms of sample s (the CF's outer-product terms).
__global__ void k_sum_terms(const float2* __restrict__ part, float2* __restrict__ vis_out, int64_t n, int rank,
                            int P) {
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
    vis_out[i] = acc;
  }
}

awg_status launch_grid(CfSetImpl* cf, PlanImpl* pl, const void* vis, const float* weight, int P, void* grid,
                       void* grid_lo, double* sumwt, int flags, cudaStream_t st) {
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  pl->last_stream = st;
  if (pl->n == 0) return AWG_OK;
  GridArgs a;
  a.rec = pl->d_rec;
  a.items = pl->d_items;
  a.class_range = pl->d_class_range;
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
  a.vis = (const float*)vis;
  a.weight = weight;
  a.grid = (float*)grid;
  a.grid_lo = (float*)grid_lo;
  a.sumwt = sumwt;
  a.sep = (const float*)cf->d_sep;
  a.sep_off = cf->d_sep_off;
  a.rank = pl->rank;
  AWG_CUDA_TRY(cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st));
  const int sms = sm_count(pl->device);
  const bool bf16 = cf->p.cf_dtype == AWG_CF_BF16;
  if (cf->separable) {
    a.class_range = pl->d_slot_range;
    for (int i = cf->slots.n - 1; i >= 0; --i) {   // largest supports first
      awg_status s = grid_slot_sep(cf->slots.S[i], i, P, a, sms, st);
      if (s != AWG_OK) return s;
    }
    return AWG_OK;
  }
  for (int c = kNumClasses - 1; c >= 0; --c) {   // largest supports first
    if (!class_present(cf, c)) continue;
    awg_status s = bf16 ? grid_class<true>(c, P, a, sms, st) : grid_class<false>(c, P, a, sms, st);
    if (s != AWG_OK) return s;
  }
  return AWG_OK;
}

awg_status launch_degrid(CfSetImpl* cf, PlanImpl* pl, const void* grid, void* vis_out, int P, cudaStream_t st) {
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  pl->last_stream = st;
  if (pl->n == 0) return AWG_OK;
  DegridArgs a;
  a.rec = pl->d_rec;
  a.items = pl->d_items;
  a.class_range = pl->d_class_range;
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
  a.grid = (const float*)grid;
  // with several terms per CF every record writes its own row of the per-term buffer, summed below
  a.vis_out = pl->rank > 1 ? (float*)pl->d_part : (float*)vis_out;
  a.sep = (const float*)cf->d_sep;
  a.sep_off = cf->d_sep_off;
  a.rank = pl->rank;
  AWG_CUDA_TRY(cudaMemsetAsync(pl->d_queue, 0, sizeof(int32_t) * kMaxSupport, st));
  const int sms = sm_count(pl->device);
  const bool bf16 = cf->p.cf_dtype == AWG_CF_BF16;
  if (cf->separable) {
    a.class_range = pl->d_slot_range;
    for (int i = cf->slots.n - 1; i >= 0; --i) {
      awg_status s = degrid_slot_sep(cf->slots.S[i], i, P, a, sms, st);
      if (s != AWG_OK) return s;
    }
  } else {
    for (int c = kNumClasses - 1; c >= 0; --c) {
      if (!class_present(cf, c)) continue;
      awg_status s = bf16 ? degrid_class<true>(c, P, a, sms, st) : degrid_class<false>(c, P, a, sms, st);
      if (s != AWG_OK) return s;
    }
  }
  if (pl->rank > 1) {   // dropped samples' rows are stale here and are zeroed next
    k_sum_terms<<<sms * 8, 256, 0, st>>>(pl->d_part, (float2*)vis_out, pl->n, pl->rank, P);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  k_zero_dropped<<<sms * 4, 256, 0, st>>>(pl->d_drop, pl->d_counters, (float*)vis_out, P);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

awg_status launch_normalize(CfSetImpl* cf, void* image, int P, const double* sumwt, int direction, cudaStream_t st) {
  if (cudaSetDevice(cf->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  const int sms = sm_count(cf->device);
  k_normalize<<<sms * 8, 256, 0, st>>>((float2*)image, cf->d_inv_taper, sumwt, cf->p.grid_n, P, direction);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

}  // namespace awg
