// PreSolvePrep (Sec. 4.1, Sec. 5.2): per-sample index math and the tiled ordering of samples.
//
// k_index   : for every (row, channel) sample, FP64 uv scaling, w-plane, CF, first tap pixel and
//             oversampling offset (the CF_ij(nu, w, t) selection of Eq. CIJ); every operation is
//             an explicitly rounded intrinsic so no multiply-add is fused; counts samples per
//             bucket, where a bucket is one (support, tile of first-tap positions).
// scan      : exclusive prefix sums over buckets (three-kernel block scan).
// k_scatter : counting-sort scatter of the kept samples into bucket order.
// k_items   : work items of at most kItemChunk samples per bucket; buckets are ordered by
//             support, so the items of each kernel class form one contiguous range.
// k_sort_items : samples of each item ordered by first-tap position (row-major; counting sort).
#include <cuda_runtime.h>

#include <algorithm>

#include "awg_internal.h"
#include "resample.cuh"

namespace awg {
namespace {

constexpr int kIndexScCache = 4096;   // channels whose f / c k_index keeps in shared memory (32 KB)

struct IndexParams {
  int64_t n;
  int rank;   // records per sample (terms per CF of a separable set)
  int C, N, OS, use_w, n_w, n_pa, n_sb, n_signed;
  double inv_dw, scale, half;
};

__device__ __forceinline__ int warp_aggregated_add(int* addr_base, int key, int amount_per_lane) {
  // Lanes with equal keys share one atomic; returns this lane's slot.
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  int base = 0;
  if (lane == leader) base = atomicAdd(addr_base + key, __popc(peers) * amount_per_lane);
  base = __shfl_sync(peers, base, leader);
  return base + rank * amount_per_lane;
}

__global__ void k_index(IndexParams ip, const double* __restrict__ uvw, const double* __restrict__ freq,
                        const int32_t* __restrict__ pa_bin, const int32_t* __restrict__ chan_sb,
                        const int32_t* __restrict__ sup_of_cf, SlotTable st, SampleRec* __restrict__ rec_tmp,
                        int32_t* __restrict__ key_out, int32_t* __restrict__ bcount, int32_t* __restrict__ drop,
                        unsigned long long* __restrict__ counters) {
  // f / c per channel, the same correctly rounded quotient for every row: formed once per block
  // in shared memory when the channels fit (kIndexScCache), else per sample
  extern __shared__ double s_sc[];
  const bool sc_cached = ip.C <= kIndexScCache;
  if (sc_cached) {
    for (int c = threadIdx.x; c < ip.C; c += blockDim.x) s_sc[c] = __ddiv_rn(freq[c], kCLight);
    __syncthreads();
  }
  unsigned long long kept = 0, taps = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ip.n; s += stride) {
    const int64_t r = s / ip.C;
    const int c = (int)(s - r * ip.C);
    const double sc = sc_cached ? s_sc[c] : __ddiv_rn(freq[c], kCLight);
    const double u = __dmul_rn(uvw[3 * r], sc);
    const double v = __dmul_rn(uvw[3 * r + 1], sc);
    const double w = __dmul_rn(uvw[3 * r + 2], sc);
    const double x = __dadd_rn(__dmul_rn(u, ip.scale), ip.half);
    const double y = __dadd_rn(__dmul_rn(v, ip.scale), ip.half);
    bool ok = isfinite(x) && isfinite(y);
    int ks = 0;
    if (ip.use_w) {
      const double k = floor(__dadd_rn(__dmul_rn(fabs(w), ip.inv_dw), 0.5));
      ok = ok && (k <= (double)(ip.n_w - 1));
      const int ki = ok ? (int)k : 0;
      ks = ip.n_w - 1 + (w < 0.0 ? -ki : ki);
    }
    int pa = 0, sb = 0;
    if (ip.n_pa > 1) {
      pa = pa_bin[r];
      if (pa < 0 || pa >= ip.n_pa) { ok = false; pa = 0; }
    }
    if (ip.n_sb > 1) {
      sb = chan_sb[c];
      if (sb < 0 || sb >= ip.n_sb) { ok = false; sb = 0; }
    }
    const int cf = (pa * ip.n_sb + sb) * ip.n_signed + ks;
    const int S = sup_of_cf[cf];
    const double hS = 0.5 * (double)S;
    const double hx = __dsub_rn(x, hS), hy = __dsub_rn(y, hS);
    const double lim = (double)(ip.N - S);
    ok = ok && (hx >= -1.0) && (hx < lim) && (hy >= -1.0) && (hy < lim);
    int key = -1;
    SampleRec rc;
    if (ok) {
      const double px = __dadd_rn(floor(hx), 1.0), py = __dadd_rn(floor(hy), 1.0);
      const double fx = __dsub_rn(px, hx), fy = __dsub_rn(py, hy);
      const double OSd = (double)ip.OS;
      const int ox = (int)floor(__dadd_rn(__dmul_rn(fx, OSd), 0.5));
      const int oy = (int)floor(__dadd_rn(__dmul_rn(fy, OSd), 0.5));
      const int p0x = (int)px, p0y = (int)py;
      rc.src = (int32_t)s;
      rc.cf = cf * ip.rank;   // term 0; term k is record s * rank + k with cf * rank + k
      rc.p0x = (uint16_t)p0x;
      rc.p0y = (uint16_t)p0y;
      rc.ox = (uint8_t)ox;
      rc.oy = (uint8_t)oy;
      rc.S = (uint8_t)S;
      rc.flags = 0;
      const int slot = st.slot_of_S[S];
      const int T = st.tile[slot];
      key = st.base[slot] + (p0y / T) * st.nt[slot] + p0x / T;
      for (int k = 0; k < ip.rank; ++k) {
        rec_tmp[s * ip.rank + k] = rc;
        rc.cf += 1;
      }
      kept += 1;
      taps += (unsigned long long)S * S;
    }
    for (int k = 0; k < ip.rank; ++k) key_out[s * ip.rank + k] = key;
    if (key >= 0) {
      warp_aggregated_add(bcount, key, ip.rank);
    } else {
      const unsigned active = __activemask();
      const unsigned peers = __match_any_sync(active, key);   // all dropping lanes
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&counters[1], (unsigned long long)__popc(peers));
      base = __shfl_sync(peers, base, leader);
      drop[base + rank] = (int32_t)s;
    }
  }
  // block reduction of the kept / taps counters
  __shared__ unsigned long long sk[32], stp[32];
  for (int o = 16; o > 0; o >>= 1) {
    kept += __shfl_xor_sync(0xffffffffu, kept, o);
    taps += __shfl_xor_sync(0xffffffffu, taps, o);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sk[wid] = kept; stp[wid] = taps; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += sk[i]; b += stp[i]; }
    if (a) atomicAdd(&counters[0], a);
    if (b) atomicAdd(&counters[2], b);
  }
}

// ---- exclusive scan of int32 [n] -> out[0..n] (out[n] = total); 1024 threads x 4 items per block
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  __shared__ int block_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
    int wi = ws;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_sums[lane] = wi - ws;
    if (lane == 31) block_total = wi;   // blockDim.x is a multiple of 32 and <= 1024
  }
  __syncthreads();
  const int res = warp_sums[wid] + inc - v;
  const int tot = block_total;
  __syncthreads();
  *total = tot;
  return res;
}

__global__ void k_scan_local(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t* __restrict__ sums,
                             int n) {
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int v[kScanItems], acc = 0;
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    acc += v[i];
  }
  int total;
  int ex = block_exclusive_scan(acc, &total);
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int32_t* sums, int nb) {
  // one block; nb <= kScanTile
  const int base = threadIdx.x * kScanItems;
  int v[kScanItems], acc = 0;
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < nb) ? sums[base + i] : 0;
    acc += v[i];
  }
  int total;
  int ex = block_exclusive_scan(acc, &total);
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < nb) sums[base + i] = ex;
    ex += v[i];
  }
  if (threadIdx.x == 0) sums[nb] = total;
}

__global__ void k_scan_add(int32_t* __restrict__ out, const int32_t* __restrict__ sums, int n, int nb) {
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  const int add = sums[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] += add;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[nb];
}

awg_status exclusive_scan(const int32_t* in, int32_t* out, int32_t* tmp, int n, cudaStream_t st) {
  const int nb = (n + kScanTile - 1) / kScanTile;
  if (nb > kScanTile) return set_error(AWG_ERR_UNSUPPORTED, "too many buckets for the scan");
  if (n == 0) {
    AWG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    return AWG_OK;
  }
  k_scan_local<<<nb, kScanThreads, 0, st>>>(in, out, tmp, n);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(tmp, nb);
  k_scan_add<<<nb, kScanThreads, 0, st>>>(out, tmp, n, nb);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(3);
  return AWG_OK;
}

__global__ void k_item_counts(const int32_t* __restrict__ boff, int32_t* __restrict__ icount, int nb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) icount[b] = (boff[b + 1] - boff[b] + kItemChunk - 1) / kItemChunk;
}

__global__ void k_items(const int32_t* __restrict__ boff, const int32_t* __restrict__ ioff, SlotTable st,
                        WorkItem* __restrict__ items, int nb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int start = boff[b], count = boff[b + 1] - start;
  if (count == 0) return;
  int slot = 0;
  while (slot + 1 < st.n && st.base[slot + 1] <= b) ++slot;
  const int local = b - st.base[slot];
  const int ty = local / st.nt[slot], tx = local - ty * st.nt[slot];
  const int S = st.S[slot];
  const int cls = class_of_support(S);
  int it = ioff[b];
  for (int j = 0; j < count; j += kItemChunk, ++it) {
    WorkItem wi;
    wi.start = start + j;
    wi.count = min(kItemChunk, count - j);
    wi.tile_x = (uint16_t)tx;
    wi.tile_y = (uint16_t)ty;
    wi.S = (uint16_t)S;
    wi.cls = (uint16_t)cls;
    items[it] = wi;
  }
}

struct ClassFirstBucket {
  int b[kNumClasses + 1];
};

__global__ void k_class_range(const int32_t* __restrict__ ioff, ClassFirstBucket fb, SlotTable st,
                              int32_t* __restrict__ range, int32_t* __restrict__ slot_range) {
  const int c = threadIdx.x;
  if (c <= kNumClasses) range[c] = ioff[fb.b[c]];
  if (c <= st.n) slot_range[c] = ioff[st.base[c]];
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ key, const SampleRec* __restrict__ rec_tmp,
                          int32_t* __restrict__ cursor, SampleRec* __restrict__ rec) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
    const int k = key[s];
    if (k < 0) continue;
    const int pos = warp_aggregated_add(cursor, k, 1);
    rec[pos] = rec_tmp[s];
  }
}

// Orders the samples of every work item by first-tap position, row-major (y, then x), with a
// counting sort in shared memory: all first taps of an item lie in one tile of at most 32 x 32
// positions, so the positions relative to the item's smallest x and y index at most kItemChunk
// bins.  Each record takes its rank in its bin (shared-memory atomic), the bin counts are scanned,
// and the records go back to the item's range in bin order (equal positions in atomic order).
// Consecutive samples then share their first-tap row for long runs and move right along it, so
// the gridding and degridding kernels recompute their row state only at row changes and a
// thread's pixels change rarely.
constexpr int kSortThreads = 256;
constexpr int kSortPer = kItemChunk / kSortThreads;   // records and bins per thread

__global__ void __launch_bounds__(kSortThreads) k_sort_items(const int32_t* __restrict__ n_items_ptr,
                                                             const WorkItem* __restrict__ items,
                                                             SampleRec* __restrict__ rec) {
  __shared__ SampleRec s_rec[kItemChunk];
  __shared__ int s_cnt[kItemChunk];
  __shared__ unsigned short s_bin[kItemChunk];
  __shared__ unsigned short s_rank[kItemChunk];
  __shared__ int s_warp[kSortThreads / 32][4];
  __shared__ int s_ext[4];
  const int n_items = *n_items_ptr;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const WorkItem wi = items[it];
    const int n = wi.count;
    // records into shared memory, with the smallest and largest first tap per axis
    int mnx = 0x7fffffff, mny = 0x7fffffff, mxx = -1, mxy = -1;
    for (int i = t; i < n; i += kSortThreads) {
      const SampleRec r = rec[wi.start + i];
      s_rec[i] = r;
      mnx = min(mnx, (int)r.p0x);
      mny = min(mny, (int)r.p0y);
      mxx = max(mxx, (int)r.p0x);
      mxy = max(mxy, (int)r.p0y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
      mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
      mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
      mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if (lane == 0) {
      s_warp[wid][0] = mnx;
      s_warp[wid][1] = mny;
      s_warp[wid][2] = mxx;
      s_warp[wid][3] = mxy;
    }
    __syncthreads();
    if (t == 0) {
      int a = 0x7fffffff, b = 0x7fffffff, c = -1, d = -1;
      for (int w = 0; w < kSortThreads / 32; ++w) {
        a = min(a, s_warp[w][0]);
        b = min(b, s_warp[w][1]);
        c = max(c, s_warp[w][2]);
        d = max(d, s_warp[w][3]);
      }
      s_ext[0] = a;
      s_ext[1] = b;
      s_ext[2] = c - a + 1;   // extent in x
      s_ext[3] = d - b + 1;   // extent in y
    }
    __syncthreads();
    const int x0 = s_ext[0], y0 = s_ext[1], ex = s_ext[2];
    const int nb = n > 0 ? ex * s_ext[3] : 0;
    if (nb > kItemChunk) {   // not one tile of at most 32 x 32 positions: leave the item as it is
      __syncthreads();
      continue;
    }
    for (int b = t; b < nb; b += kSortThreads) s_cnt[b] = 0;
    __syncthreads();
    for (int i = t; i < n; i += kSortThreads) {
      const int b = ((int)s_rec[i].p0y - y0) * ex + ((int)s_rec[i].p0x - x0);
      s_bin[i] = (unsigned short)b;
      s_rank[i] = (unsigned short)atomicAdd(&s_cnt[b], 1);
    }
    __syncthreads();
    // exclusive scan of the bin counts: kSortPer consecutive bins per thread, then the threads
    int v[kSortPer];
    int run = 0;
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
      const int b = t * kSortPer + k;
      v[k] = b < nb ? s_cnt[b] : 0;
      run += v[k];
    }
    int incl = run;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid][0] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += s_warp[w][0];
    int off = before + incl - run;
#pragma unroll
    for (int k = 0; k < kSortPer; ++k) {
      const int b = t * kSortPer + k;
      if (b < nb) s_cnt[b] = off;
      off += v[k];
    }
    __syncthreads();
    for (int i = t; i < n; i += kSortThreads) rec[wi.start + s_cnt[s_bin[i]] + s_rank[i]] = s_rec[i];
    __syncthreads();
  }
}

struct PhaseArgs {
  const double* uvw;
  const double* freq;
  const double* row_dlm;
  int C;
  double dl, dm, dn;
};

__global__ void k_phasors(PhaseArgs a, int64_t n, float2* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) out[s] = phasor_of(a, (int)s);
}

}  // namespace

awg_status compute_phasors(PlanImpl* pl, cudaStream_t st) {
  if (pl->n == 0) return AWG_OK;
  PhaseArgs a{pl->d_uvw, pl->d_freq, pl->d_row_dlm, pl->C, pl->dl, pl->dm, pl->dn};
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
  const int blocks = (int)std::min<int64_t>((pl->n + 255) / 256, (int64_t)std::max(sms, 1) * 8);
  k_phasors<<<blocks, 256, 0, st>>>(a, pl->n, pl->d_phasor);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// class_of_support is also used in device code above.
awg_status plan_build(PlanImpl* pl, const double* uvw, const double* freq, const int32_t* pa_bin,
                      const int32_t* chan_sb, cudaStream_t st) {
  CfSetImpl* cf = pl->cf;
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  pl->last_stream = st;
  if (pl->has_phase && pl->n > 0) {
    AWG_CUDA_TRY(cudaMemcpyAsync(pl->d_uvw, uvw, sizeof(double) * 3 * pl->R, cudaMemcpyDeviceToDevice, st));
    AWG_CUDA_TRY(cudaMemcpyAsync(pl->d_freq, freq, sizeof(double) * pl->C, cudaMemcpyDeviceToDevice, st));
    awg_status ps = compute_phasors(pl, st);
    if (ps != AWG_OK) return ps;
  }
  const int nb = pl->n_buckets;
  AWG_CUDA_TRY(cudaMemsetAsync(pl->d_bcount, 0, sizeof(int32_t) * (nb + 1), st));
  AWG_CUDA_TRY(cudaMemsetAsync(pl->d_counters, 0, 4 * sizeof(unsigned long long), st));
  IndexParams ip;
  ip.n = pl->n;
  ip.rank = pl->rank;
  ip.C = pl->C;
  ip.N = cf->p.grid_n;
  ip.OS = cf->p.oversampling;
  ip.use_w = cf->p.use_w;
  ip.n_w = cf->p.use_w ? cf->p.n_wplanes : 1;
  ip.n_pa = cf->p.n_pa_bins;
  ip.n_sb = cf->p.n_subbands;
  ip.n_signed = cf->n_signed;
  ip.inv_dw = cf->p.use_w ? (double)(cf->p.n_wplanes - 1) / cf->p.w_max_lambda : 0.0;
  ip.scale = (double)cf->p.grid_n * cf->p.cell_rad;
  ip.half = (double)(cf->p.grid_n / 2);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device);
  if (pl->n > 0) {
    const int blocks = (int)std::min<int64_t>((pl->n + 255) / 256, (int64_t)sms * 8);
    const size_t sc_bytes = ip.C <= kIndexScCache ? sizeof(double) * (size_t)ip.C : 0;
    k_index<<<blocks, 256, sc_bytes, st>>>(ip, uvw, freq, pa_bin, chan_sb, cf->d_sup, cf->slots, pl->d_rec_tmp, pl->d_key,
                                    pl->d_bcount, pl->d_drop, pl->d_counters);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  awg_status s = exclusive_scan(pl->d_bcount, pl->d_boff, pl->d_scan_tmp, nb, st);
  if (s != AWG_OK) return s;
  if (nb > 0) {
    k_item_counts<<<(nb + 255) / 256, 256, 0, st>>>(pl->d_boff, pl->d_icount, nb);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  s = exclusive_scan(pl->d_icount, pl->d_ioff, pl->d_scan_tmp, nb, st);
  if (s != AWG_OK) return s;
  if (nb > 0) {
    k_items<<<(nb + 255) / 256, 256, 0, st>>>(pl->d_boff, pl->d_ioff, cf->slots, pl->d_items, nb);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  ClassFirstBucket fb;
  for (int c = 0; c <= kNumClasses; ++c) {
    fb.b[c] = nb;
    for (int i = 0; i < cf->slots.n; ++i)
      if (class_of_support(cf->slots.S[i]) >= c) { fb.b[c] = cf->slots.base[i]; break; }
  }
  k_class_range<<<1, kMaxSupport + 1, 0, st>>>(pl->d_ioff, fb, cf->slots, pl->d_class_range, pl->d_slot_range);
  AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  if (pl->n > 0 && nb > 0) {
    AWG_CUDA_TRY(cudaMemcpyAsync(pl->d_bcount, pl->d_boff, sizeof(int32_t) * nb, cudaMemcpyDeviceToDevice, st));
    const int blocks = (int)std::min<int64_t>((pl->n_rec + 255) / 256, (int64_t)sms * 8);
    k_scatter<<<blocks, 256, 0, st>>>(pl->n_rec, pl->d_key, pl->d_rec_tmp, pl->d_bcount, pl->d_rec);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    k_sort_items<<<sms * 8, kSortThreads, 0, st>>>(pl->d_ioff + nb, pl->d_items, pl->d_rec);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  return AWG_OK;
}

}  // namespace awg
