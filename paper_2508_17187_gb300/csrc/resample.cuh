// Gridding (G, Eq. IMAGE-MOD) and degridding (D, Eq. ME-MOD-GRIDDED) kernels for sm_103a.
//
// Work decomposition (both directions): a work item is up to kItemChunk samples of one support S
// whose first tap lies in one TILE x TILE block of the grid, so every tap of the item falls in a
// U x U window, U = TILE + S - 1.  Each CTA is persistent and pulls items from a per-class queue.
//
// Gridding: the window lives in shared memory.  Thread t owns the tap residues r = t + k NT
// (r < S^2, (rx, ry) = (r mod S, r div S)); for a sample with first tap p0 the residue touches
// the unique pixel p0 + ((r - p0) mod S) of its footprint.  Consecutive samples of an item start
// close together, so the pixel of a residue changes rarely: the thread accumulates
// conj(c) * w * V for all P pols in registers and adds the registers into the shared window only
// when the pixel changes (no two residues share a pixel, so no shared atomics are needed).  At
// the end of the item each window pixel is flushed to the global grid with one vector atomic.
//
// Degridding: the window of the grid is loaded into shared memory once per item.  For a batch of
// B = 32 / (2P) samples every thread forms its residues' partial sums sum c * grid for each
// sample and pol; one warp butterfly reduce-scatter leaves component `lane` of the batch in lane
// `lane`, the warps' results are summed through shared memory and written as whole samples.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "awg_internal.h"

namespace awg {

constexpr int kStage = 32;   // samples staged in shared memory at a time

struct GridArgs {
  const SampleRec* rec;
  const WorkItem* items;
  const int32_t* class_range;
  int32_t* queue;
  const void* cf;
  const int64_t* cf_off;
  int OS, N, C, flags, has_phase;
  double dl, dm, dn;
  const double* uvw;
  const double* freq;
  const double* row_dlm; // per-row (dl, dm) [R][2] or NULL (then dl, dm, dn apply to every row)
  const float2* phasor;  // per-sample phasor [n] formed by the plan, or NULL (no phase term)
  const float* vis;      // interleaved c64 [n][P]
  const float* weight;   // [n][P]
  float* grid;           // c64 [N][N][P] (or complex128 with AWG_GRID_FP64)
  float* grid_lo;        // c64 [N][N][P] with AWG_GRID_KAHAN
  double* sumwt;         // [P]
  const float* sep;      // separable CF factors (c64), or NULL
  const int64_t* sep_off;
  int n_sep_off;         // entries of sep_off
  int rank;              // records per sample; only term 0 (cf % rank == 0) adds its weight
  // Mueller element launches (separable kernels): factor offsets at sep_off[cf_shift + rc.cf];
  // sample s reads vis / weight at s vstride + voff and pixel i of the grid is i gstride + goff
  // (P pols from there); otherwise cf_shift = 0, vstride = gstride = P, voff = goff = 0.
  int64_t cf_shift;
  int vstride, voff, gstride, goff;
  // Full-polarisation base passes (fused separable kernels, P = 4): when mix != NULL the kernel
  // grids u_q = sum_p mix[4 q + p] w_p V_p as pol q instead of w_q V_q; only the pols set in pmask
  // add their weights to sumwt.  Otherwise mix = NULL and pmask has all P bits set.
  const float2* mix;
  int pmask;
  unsigned long long* err;   // error word of the launch (a bounded wait that gave up), or NULL
  int withhold;              // test hook (awg_debug_ws_withhold): withhold the first chunk's hand-over
};

struct DegridArgs {
  const SampleRec* rec;
  const WorkItem* items;
  const int32_t* class_range;
  int32_t* queue;
  const void* cf;
  const int64_t* cf_off;
  int OS, N, C, has_phase;
  double dl, dm, dn;
  const double* uvw;
  const double* freq;
  const double* row_dlm; // per-row (dl, dm) [R][2] or NULL
  const float2* phasor;  // per-sample phasor [n] formed by the plan, or NULL
  const float* grid;     // c64 [N][N][P]
  float* vis_out;        // c64 [n][P]; with rank > 1 the per-term values [n][rank][P]
  const float* sep;      // separable CF factors (c64), or NULL
  const int64_t* sep_off;
  int n_sep_off;         // entries of sep_off
  int rank;              // records per sample (term k of sample s writes vis_out row s * rank + k)
  int64_t cf_shift;      // as in GridArgs; the output row r goes to vis_out at r vstride + voff,
  int vstride, voff, gstride, goff;
  int accumulate;        // 0: write vis_out, 1: add to it, -1: subtract from it (residuals)
  // Full-polarisation base passes (fused separable kernels, P = 4): with Y_q the CF applied to
  // grid pol q, output pol p = sum_q mix[4 p + q] Y_q when mix != NULL (else Y_p); only the pols
  // set in pmask are written.
  const float2* mix;
  int pmask;
  unsigned long long* err;   // error word of the launch (a bounded wait that gave up), or NULL
  int withhold;              // test hook (awg_debug_ws_withhold): withhold the first chunk's hand-over
};

template <bool BF16>
__device__ __forceinline__ float2 ld_cf(const void* base, long long i);

template <>
__device__ __forceinline__ float2 ld_cf<false>(const void* base, long long i) {
  return __ldg(reinterpret_cast<const float2*>(base) + i);
}

template <>
__device__ __forceinline__ float2 ld_cf<true>(const void* base, long long i) {
  const unsigned int raw = __ldg(reinterpret_cast<const unsigned int*>(base) + i);
  __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&raw);
  return __bfloat1622float2(h);
}

// exp(+2 pi i (u dl + v dm + w dn)) for sample src; argument in FP64 turns, reduced before the
// FP32 sine and cosine (the phase-gradient term of Eq. CIJ).
__device__ __forceinline__ float2 sample_phasor(const double* uvw, const double* freq, int C, int src, double dl,
                                                double dm, double dn) {
  const int r = src / C, c = src - (src / C) * C;
  const double sc = freq[c] / kCLight;
  double t = (uvw[3 * r] * sc) * dl + (uvw[3 * r + 1] * sc) * dm + (uvw[3 * r + 2] * sc) * dn;
  t -= rint(t);
  float s, co;
  sincospif(2.0f * (float)t, &s, &co);
  return make_float2(co, s);
}

// Per-row phase centres (mosaic pointings, antenna pointing offsets): row r of the plan has its
// own (dl, dm) at row_dlm[2 r], and dn = sqrt(1 - dl^2 - dm^2) - 1 in a cancellation-free form.
template <class Args>
__device__ __forceinline__ float2 phasor_of(const Args& a, int src) {
  if (a.row_dlm) {
    const int r = src / a.C;
    const double dl = a.row_dlm[2 * r], dm = a.row_dlm[2 * r + 1];
    const double q = dl * dl + dm * dm;
    return sample_phasor(a.uvw, a.freq, a.C, src, dl, dm, -q / (1.0 + sqrt(1.0 - q)));
  }
  return sample_phasor(a.uvw, a.freq, a.C, src, a.dl, a.dm, a.dn);
}

template <int SMAX, int TILE, int P>
struct GridLayout {
  static constexpr int UMAX = TILE + SMAX - 1;
  static constexpr size_t tile_bytes = (size_t)UMAX * UMAX * P * sizeof(float2);
  static constexpr size_t bytes = tile_bytes + kStage * (P * sizeof(float2) + sizeof(long long) + sizeof(int));
};

// Add the P pols of one window pixel into the global grid; g is the complex-element index of
// pol 0 of the pixel ((y N + x) P), so the pixel's floats start at 2 g.
template <int P>
__device__ __forceinline__ void flush_pixel(const GridArgs& a, size_t g, const float2 (&v)[P]) {
  if (a.flags & AWG_GRID_FP64) {
    double* d = reinterpret_cast<double*>(a.grid) + 2 * g;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      atomicAdd(d + 2 * p, (double)v[p].x);
      atomicAdd(d + 2 * p + 1, (double)v[p].y);
    }
    return;
  }
  float* dst = a.grid + 2 * g;
  if (!(a.flags & AWG_GRID_KAHAN)) {
    // plain flush: the old value is never read, so these compile to reductions (no return trip)
    if constexpr (P == 1) {
      atomicAdd(reinterpret_cast<float2*>(dst), v[0]);
    } else {
#pragma unroll
      for (int h = 0; h < P / 2; ++h)
        atomicAdd(reinterpret_cast<float4*>(dst + 4 * h),
                  make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y));
    }
    return;
  }
  // compensated flush: TwoSum of the value the atomic saw and the added value
  if constexpr (P == 1) {
    const float2 old = atomicAdd(reinterpret_cast<float2*>(dst), v[0]);
    const float s0 = old.x + v[0].x, s1 = old.y + v[0].y;
    const float b0 = s0 - old.x, b1 = s1 - old.y;
    const float2 e = make_float2((old.x - (s0 - b0)) + (v[0].x - b0), (old.y - (s1 - b1)) + (v[0].y - b1));
    if (e.x != 0.f || e.y != 0.f) atomicAdd(reinterpret_cast<float2*>(a.grid_lo + 2 * g), e);
  } else {
#pragma unroll
    for (int h = 0; h < P / 2; ++h) {
      const float4 val = make_float4(v[2 * h].x, v[2 * h].y, v[2 * h + 1].x, v[2 * h + 1].y);
      const float4 old = atomicAdd(reinterpret_cast<float4*>(dst + 4 * h), val);
      const float o[4] = {old.x, old.y, old.z, old.w};
      const float b[4] = {val.x, val.y, val.z, val.w};
      float e[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float s = o[q] + b[q];
        const float bb = s - o[q];
        e[q] = (o[q] - (s - bb)) + (b[q] - bb);
      }
      if (e[0] != 0.f || e[1] != 0.f || e[2] != 0.f || e[3] != 0.f)
        atomicAdd(reinterpret_cast<float4*>(a.grid_lo + 2 * g + 4 * h), make_float4(e[0], e[1], e[2], e[3]));
    }
  }
}

template <int SMAX, int NT, int TILE, int P, bool BF16>
__global__ void __launch_bounds__(NT) k_grid(const GridArgs a, const int cls) {
  constexpr int R = (SMAX * SMAX + NT - 1) / NT;
  using L = GridLayout<SMAX, TILE, P>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float2* s_a = reinterpret_cast<float2*>(smem + L::tile_bytes);
  long long* s_slice = reinterpret_cast<long long*>(s_a + kStage * P);
  int* s_pack = reinterpret_cast<int*>(s_slice + kStage);
  __shared__ int s_item;
  __shared__ double s_wsum[NT / 32][P];

  const int tid = threadIdx.x;
  const int begin = a.class_range[cls], end = a.class_range[cls + 1];
  double wsum[P];
#pragma unroll
  for (int p = 0; p < P; ++p) wsum[p] = 0.0;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = begin + atomicAdd(a.queue + cls, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= end) break;
    const WorkItem wi = a.items[it];
    const int S = wi.S, SS = S * S, U = TILE + S - 1;
    const int X0 = wi.tile_x * TILE, Y0 = wi.tile_y * TILE;
    for (int i = tid; i < U * U * P; i += NT) tile[i] = make_float2(0.f, 0.f);
    int rxy[R], cur[R];
    float2 acc[R][P];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = tid + k * NT;
      rxy[k] = (r < SS) ? ((r % S) | ((r / S) << 8)) : -1;
      cur[k] = -1;
#pragma unroll
      for (int p = 0; p < P; ++p) acc[k][p] = make_float2(0.f, 0.f);
    }
    for (int c0 = 0; c0 < wi.count; c0 += kStage) {
      const int nst = min(kStage, wi.count - c0);
      __syncthreads();
      if (tid < nst) {
        const SampleRec rc = a.rec[wi.start + c0 + tid];
        const float* vp = a.vis + (size_t)rc.src * 2 * P;
        const float* wp = a.weight + (size_t)rc.src * P;
        float2 v[P];
        float wt[P];
        if (P == 4) {
          const float4 v0 = __ldg(reinterpret_cast<const float4*>(vp));
          const float4 v1 = __ldg(reinterpret_cast<const float4*>(vp) + 1);
          const float4 w4 = __ldg(reinterpret_cast<const float4*>(wp));
          v[0] = make_float2(v0.x, v0.y); v[1 % P] = make_float2(v0.z, v0.w);
          v[2 % P] = make_float2(v1.x, v1.y); v[3 % P] = make_float2(v1.z, v1.w);
          wt[0] = w4.x; wt[1 % P] = w4.y; wt[2 % P] = w4.z; wt[3 % P] = w4.w;
        } else if (P == 2) {
          const float4 v0 = __ldg(reinterpret_cast<const float4*>(vp));
          const float2 w2 = __ldg(reinterpret_cast<const float2*>(wp));
          v[0] = make_float2(v0.x, v0.y); v[1 % P] = make_float2(v0.z, v0.w);
          wt[0] = w2.x; wt[1 % P] = w2.y;
        } else {
          v[0] = __ldg(reinterpret_cast<const float2*>(vp));
          wt[0] = __ldg(wp);
        }
        float2 ph = make_float2(1.f, 0.f);
        if (a.phasor) ph = a.phasor[rc.src];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          wsum[p] += (double)wt[p];
          const float xr = wt[p] * v[p].x, xi = wt[p] * v[p].y;
          s_a[tid * P + p] = make_float2(xr * ph.x - xi * ph.y, xr * ph.y + xi * ph.x);
        }
        s_slice[tid] = a.cf_off[rc.cf] + (long long)(rc.oy * (a.OS + 1) + rc.ox) * SS;
        s_pack[tid] = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | ((rc.p0x % S) << 16) | ((rc.p0y % S) << 24);
      }
      __syncthreads();
      for (int j = 0; j < nst; ++j) {
        const int pk = s_pack[j];
        const int dx = pk & 0xff, dy = (pk >> 8) & 0xff, mx = (pk >> 16) & 0xff, my = (pk >> 24) & 0xff;
        const long long sl = s_slice[j];
        float2 av[P];
#pragma unroll
        for (int p = 0; p < P; ++p) av[p] = s_a[j * P + p];
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (rxy[k] >= 0) {
            int tx = (rxy[k] & 0xff) - mx;
            tx += (tx < 0) ? S : 0;
            int ty = (rxy[k] >> 8) - my;
            ty += (ty < 0) ? S : 0;
            const int lp = (ty + dy) * U + (tx + dx);
            if (lp != cur[k]) {
              if (cur[k] >= 0) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                  float2* t = tile + cur[k] * P + p;
                  t->x += acc[k][p].x;
                  t->y += acc[k][p].y;
                  acc[k][p] = make_float2(0.f, 0.f);
                }
              }
              cur[k] = lp;
            }
            const float2 c = ld_cf<BF16>(a.cf, sl + ty * S + tx);
#pragma unroll
            for (int p = 0; p < P; ++p) {
              acc[k][p].x = fmaf(c.x, av[p].x, fmaf(c.y, av[p].y, acc[k][p].x));
              acc[k][p].y = fmaf(c.x, av[p].y, fmaf(-c.y, av[p].x, acc[k][p].y));
            }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (cur[k] >= 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          float2* t = tile + cur[k] * P + p;
          t->x += acc[k][p].x;
          t->y += acc[k][p].y;
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < U * U; i += NT) {
      const int ly = i / U, lx = i - ly * U;
      const int gy = Y0 + ly, gx = X0 + lx;
      if (gy >= a.N || gx >= a.N) continue;
      float2 v[P];
      bool nz = false;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        v[p] = tile[i * P + p];
        nz |= (v[p].x != 0.f) || (v[p].y != 0.f);
      }
      if (nz) flush_pixel<P>(a, ((size_t)gy * a.N + gx) * P, v);   // complex-element index of pol 0
    }
  }
  // sum of weights: warp, then block, then one FP64 atomic per pol
  const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double v = wsum[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_wsum[wid][p] = v;
  }
  __syncthreads();
  if (tid < P) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += s_wsum[w][tid];
    if (v != 0.0) atomicAdd(a.sumwt + tid, v);
  }
}

template <int SMAX, int TILE, int P>
struct DegridLayout {
  static constexpr int UMAX = TILE + SMAX - 1;
  static constexpr size_t tile_bytes = (size_t)UMAX * UMAX * P * sizeof(float2);
  static constexpr size_t bytes =
      tile_bytes + kStage * (sizeof(long long) + sizeof(int) + sizeof(int) + sizeof(float2));
};

template <int SMAX, int NT, int TILE, int P, bool BF16>
__global__ void __launch_bounds__(NT) k_degrid(const DegridArgs a, const int cls) {
  constexpr int R = (SMAX * SMAX + NT - 1) / NT;
  constexpr int NW = NT / 32;
  constexpr int B = 32 / (2 * P);     // samples per reduction batch
  using L = DegridLayout<SMAX, TILE, P>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  long long* s_slice = reinterpret_cast<long long*>(smem + L::tile_bytes);
  int* s_pack = reinterpret_cast<int*>(s_slice + kStage);
  int* s_src = s_pack + kStage;
  float2* s_ph = reinterpret_cast<float2*>(s_src + kStage);
  __shared__ float s_red[2][NW][32];
  __shared__ int s_item;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int begin = a.class_range[cls], end = a.class_range[cls + 1];
  int buf = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = begin + atomicAdd(a.queue + cls, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= end) break;
    const WorkItem wi = a.items[it];
    const int S = wi.S, SS = S * S, U = TILE + S - 1;
    const int X0 = wi.tile_x * TILE, Y0 = wi.tile_y * TILE;
    for (int i = tid; i < U * U; i += NT) {
      const int ly = i / U, lx = i - ly * U;
      const int gy = Y0 + ly, gx = X0 + lx;
      const bool in = gy < a.N && gx < a.N;
      const float* src = a.grid + ((size_t)gy * a.N + gx) * 2 * P;
      if (P == 4) {
        const float4 g0 = in ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 g1 = in ? __ldg(reinterpret_cast<const float4*>(src) + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(tile + i * P)[0] = g0;
        reinterpret_cast<float4*>(tile + i * P)[1] = g1;
      } else if (P == 2) {
        const float4 g0 = in ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(tile + i * P)[0] = g0;
      } else {
        tile[i] = in ? __ldg(reinterpret_cast<const float2*>(src)) : make_float2(0.f, 0.f);
      }
    }
    int rxy[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = tid + k * NT;
      rxy[k] = (r < SS) ? ((r % S) | ((r / S) << 8)) : -1;
    }
    for (int c0 = 0; c0 < wi.count; c0 += kStage) {
      const int nst = min(kStage, wi.count - c0);
      __syncthreads();
      if (tid < nst) {
        const SampleRec rc = a.rec[wi.start + c0 + tid];
        s_slice[tid] = a.cf_off[rc.cf] + (long long)(rc.oy * (a.OS + 1) + rc.ox) * SS;
        s_pack[tid] = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | ((rc.p0x % S) << 16) | ((rc.p0y % S) << 24);
        s_src[tid] = rc.src;
        float2 ph = make_float2(1.f, 0.f);
        if (a.phasor) ph = a.phasor[rc.src];
        s_ph[tid] = ph;
      }
      __syncthreads();
      for (int j0 = 0; j0 < nst; j0 += B) {
        float vals[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) vals[q] = 0.f;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int j = j0 + b;
          if (j < nst) {
            const int pk = s_pack[j];
            const int dx = pk & 0xff, dy = (pk >> 8) & 0xff, mx = (pk >> 16) & 0xff, my = (pk >> 24) & 0xff;
            const long long sl = s_slice[j];
#pragma unroll
            for (int k = 0; k < R; ++k) {
              if (rxy[k] >= 0) {
                int tx = (rxy[k] & 0xff) - mx;
                tx += (tx < 0) ? S : 0;
                int ty = (rxy[k] >> 8) - my;
                ty += (ty < 0) ? S : 0;
                const int lp = (ty + dy) * U + (tx + dx);
                const float2 c = ld_cf<BF16>(a.cf, sl + ty * S + tx);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                  const float2 g = tile[lp * P + p];
                  vals[b * 2 * P + 2 * p] = fmaf(c.x, g.x, fmaf(-c.y, g.y, vals[b * 2 * P + 2 * p]));
                  vals[b * 2 * P + 2 * p + 1] = fmaf(c.x, g.y, fmaf(c.y, g.x, vals[b * 2 * P + 2 * p + 1]));
                }
              }
            }
          }
        }
        // butterfly reduce-scatter: afterwards lane L holds the warp sum of component L
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          const bool upper = (lane & off) != 0;
#pragma unroll
          for (int i = 0; i < off; ++i) {
            const float send = upper ? vals[i] : vals[i + off];
            const float keep = upper ? vals[i + off] : vals[i];
            vals[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
          }
        }
        s_red[buf][wid][lane] = vals[0];
        __syncthreads();
        if (wid == 0) {
          float v = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) v += s_red[buf][w][lane];
          const int b = lane / (2 * P), comp = lane - b * 2 * P;
          const int j = j0 + b;
          const float partner = __shfl_xor_sync(0xffffffffu, v, 1);
          if (j < nst) {
            const float2 ph = s_ph[j];   // multiply by conj(phasor)
            const float out = (comp & 1) ? (v * ph.x - partner * ph.y) : (v * ph.x + partner * ph.y);
            float* o = a.vis_out + (size_t)s_src[j] * 2 * P + comp;
            *o = a.accumulate == 0 ? out : a.accumulate > 0 ? *o + out : *o - out;
          }
        }
        buf ^= 1;
      }
    }
  }
}

__global__ void k_zero_dropped(const int32_t* __restrict__ drop, const unsigned long long* __restrict__ counters,
                               float* __restrict__ vis_out, int P);

template <int CLS, int P, bool BF16>
awg_status run_grid(const GridArgs& a, int sms, cudaStream_t st) {
  constexpr ClassCfg cc = kClasses[CLS];
  using L = GridLayout<cc.smax, cc.tile, P>;
  auto kern = k_grid<cc.smax, cc.nt, cc.tile, P, BF16>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cc.nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "gridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, cc.nt, L::bytes, st>>>(a, CLS);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

template <int CLS, int P, bool BF16>
awg_status run_degrid(const DegridArgs& a, int sms, cudaStream_t st) {
  constexpr ClassCfg cc = kClasses[CLS];
  using L = DegridLayout<cc.smax, cc.tile, P>;
  auto kern = k_degrid<cc.smax, cc.nt, cc.tile, P, BF16>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cc.nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "degridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, cc.nt, L::bytes, st>>>(a, CLS);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// Per-translation-unit instantiation lists (grid_*.cu / degrid_*.cu).
#define AWG_FOR_CLASSES_AND_POLS(M, BF) \
  M(0, 1, BF) M(0, 2, BF) M(0, 4, BF) M(1, 1, BF) M(1, 2, BF) M(1, 4, BF) M(2, 1, BF) M(2, 2, BF) M(2, 4, BF) \
  M(3, 1, BF) M(3, 2, BF) M(3, 4, BF) M(4, 1, BF) M(4, 2, BF) M(4, 4, BF) M(5, 1, BF) M(5, 2, BF) M(5, 4, BF)

#define AWG_DECLARE_GRID(C, P, BF) extern template awg_status run_grid<C, P, BF>(const GridArgs&, int, cudaStream_t);
#define AWG_DECLARE_DEGRID(C, P, BF) \
  extern template awg_status run_degrid<C, P, BF>(const DegridArgs&, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID(C, P, BF) template awg_status run_grid<C, P, BF>(const GridArgs&, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID(C, P, BF) \
  template awg_status run_degrid<C, P, BF>(const DegridArgs&, int, cudaStream_t);

}  // namespace awg
