// Gridding and degridding with separable CFs, c[oy][ox][ty][tx] = fy[oy][ty] * fx[ox][tx].
//
// PS and W-projection CFs are outer products to FP32 precision (the W screen's non-separable
// part is below 1e-7 of the peak for fields of a fraction of a degree), so a sample needs only
// its two factor rows (2 S values) instead of an S x S slice.  The work decomposition is that of
// resample.cuh; the tap ownership is arranged so the factorisation also saves arithmetic:
//
// Thread t of NT owns column residue rx = t mod S and rows ry = t div S + k G, G = NT div S
// (threads t >= G S idle).  Gridding: per sample the thread forms alpha_p = conj(fx[tx]) w V_p
// once for its column and then adds conj(fy[ty]) alpha_p for each of its rows: 4 FFMA per tap
// and pol, as with a full table, but the only per-tap load is fy[ty] from shared memory.
// Registers accumulate until a residue's pixel changes (column change: all rows; row change:
// that row); then they are added into the shared window, which is flushed with one vector
// atomic per pixel at the end of the item.
// Degridding: per sample the thread sums fy[ty] grid[Y][X][p] over its rows and multiplies by
// fx[tx] once; a warp reduce-scatter and a shared-memory pass finish the sum as in resample.cuh.
#pragma once

#include "resample.cuh"

namespace awg {

constexpr int kSepStage = 16;   // samples staged per chunk (their factor rows live in shared memory)

// Rows per thread needed by any support of a class: max over S in (smin, smax] of ceil(S / (NT / S)).
__host__ __device__ constexpr int sep_rows(int smin, int smax, int nt) {
  int r = 1;
  for (int S = smin + 1; S <= smax; ++S) {
    const int G = nt / S;
    const int rows = (S + G - 1) / G;
    r = rows > r ? rows : r;
  }
  return r;
}

template <int SMAX, int TILE, int P>
struct SepLayout {
  static constexpr int UMAX = TILE + SMAX - 1;
  static constexpr size_t tile_bytes = (size_t)UMAX * UMAX * P * sizeof(float2);
  static constexpr size_t f_bytes = (size_t)kSepStage * 2 * SMAX * sizeof(float2);
  static constexpr size_t a_bytes = (size_t)kSepStage * P * sizeof(float2);
  static constexpr size_t bytes = tile_bytes + f_bytes + a_bytes + kSepStage * (2 * sizeof(long long) + 4 * sizeof(int));
};

template <int SMIN, int SMAX, int NT, int TILE, int P>
__global__ void __launch_bounds__(NT) k_grid_sep(const GridArgs a, const int cls) {
  constexpr int R = sep_rows(SMIN, SMAX, NT);
  using L = SepLayout<SMAX, TILE, P>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float2* s_f = reinterpret_cast<float2*>(smem + L::tile_bytes);              // [stage][2][SMAX]
  float2* s_a = reinterpret_cast<float2*>(smem + L::tile_bytes + L::f_bytes);  // [stage][P]
  long long* s_fxo = reinterpret_cast<long long*>(smem + L::tile_bytes + L::f_bytes + L::a_bytes);
  long long* s_fyo = s_fxo + kSepStage;
  int* s_pack = reinterpret_cast<int*>(s_fyo + kSepStage);
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
    const int S = wi.S, U = TILE + S - 1;
    const int X0 = wi.tile_x * TILE, Y0 = wi.tile_y * TILE;
    const int G = NT / S;
    const bool active = tid < G * S;
    const int rx = tid % S, ry0 = tid / S;
    for (int i = tid; i < U * U * P; i += NT) tile[i] = make_float2(0.f, 0.f);
    int curX = -1;
    int curY[R];
    float2 acc[R][P];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      curY[k] = -1;
#pragma unroll
      for (int p = 0; p < P; ++p) acc[k][p] = make_float2(0.f, 0.f);
    }
    for (int c0 = 0; c0 < wi.count; c0 += kSepStage) {
      const int nst = min(kSepStage, wi.count - c0);
      __syncthreads();
      if (tid < nst) {
        const SampleRec rc = a.rec[wi.start + c0 + tid];
        const float* vp = a.vis + (size_t)rc.src * 2 * P;
        const float* wp = a.weight + (size_t)rc.src * P;
        float2 v[P];
        float wt[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          v[p] = __ldg(reinterpret_cast<const float2*>(vp) + p);
          wt[p] = __ldg(wp + p);
        }
        float2 ph = make_float2(1.f, 0.f);
        if (a.has_phase) ph = sample_phasor(a.uvw, a.freq, a.C, rc.src, a.dl, a.dm, a.dn);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          wsum[p] += (double)wt[p];
          const float xr = wt[p] * v[p].x, xi = wt[p] * v[p].y;
          s_a[tid * P + p] = make_float2(xr * ph.x - xi * ph.y, xr * ph.y + xi * ph.x);
        }
        const long long base = a.sep_off[rc.cf];
        s_fxo[tid] = base + (long long)rc.ox * S;
        s_fyo[tid] = base + (long long)(a.OS + 1) * S + (long long)rc.oy * S;
        s_pack[tid] = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | ((rc.p0x % S) << 16) | ((rc.p0y % S) << 24);
      }
      __syncthreads();
      for (int i = tid; i < nst * 2 * S; i += NT) {
        const int j = i / (2 * S), r = i - j * 2 * S;
        const long long src = r < S ? s_fxo[j] + r : s_fyo[j] + (r - S);
        s_f[(j * 2 + (r < S ? 0 : 1)) * SMAX + (r < S ? r : r - S)] =
            __ldg(reinterpret_cast<const float2*>(a.sep) + src);
      }
      __syncthreads();
      if (active) {
        for (int j = 0; j < nst; ++j) {
          const int pk = s_pack[j];
          const int dx = pk & 0xff, dy = (pk >> 8) & 0xff, mx = (pk >> 16) & 0xff, my = (pk >> 24) & 0xff;
          int tx = rx - mx;
          tx += (tx < 0) ? S : 0;
          const int X = dx + tx;
          const float2 fxv = s_f[(j * 2) * SMAX + tx];
          float2 al[P];
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const float2 av = s_a[j * P + p];
            al[p] = make_float2(fxv.x * av.x + fxv.y * av.y, fxv.x * av.y - fxv.y * av.x);   // conj(fx) a
          }
          if (X != curX) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
              if (curY[k] >= 0) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                  float2* t = tile + (curY[k] * U + curX) * P + p;
                  t->x += acc[k][p].x;
                  t->y += acc[k][p].y;
                  acc[k][p] = make_float2(0.f, 0.f);
                }
                curY[k] = -1;
              }
            }
            curX = X;
          }
          int ty0 = ry0 - my;
          ty0 += (ty0 < 0) ? S : 0;
          const float2* fyrow = s_f + (j * 2 + 1) * SMAX;
#pragma unroll
          for (int k = 0; k < R; ++k) {
            if (ry0 + k * G < S) {
              int ty = ty0 + k * G;
              ty -= (ty >= S) ? S : 0;
              const int Y = dy + ty;
              if (Y != curY[k]) {
                if (curY[k] >= 0) {
#pragma unroll
                  for (int p = 0; p < P; ++p) {
                    float2* t = tile + (curY[k] * U + curX) * P + p;
                    t->x += acc[k][p].x;
                    t->y += acc[k][p].y;
                    acc[k][p] = make_float2(0.f, 0.f);
                  }
                }
                curY[k] = Y;
              }
              const float2 f = fyrow[ty];
#pragma unroll
              for (int p = 0; p < P; ++p) {   // acc += conj(fy) alpha
                acc[k][p].x = fmaf(f.x, al[p].x, fmaf(f.y, al[p].y, acc[k][p].x));
                acc[k][p].y = fmaf(f.x, al[p].y, fmaf(-f.y, al[p].x, acc[k][p].y));
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (curY[k] >= 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          float2* t = tile + (curY[k] * U + curX) * P + p;
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
      if (nz) flush_pixel<P>(a, ((size_t)gy * a.N + gx) * P, v);
    }
  }
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

template <int SMIN, int SMAX, int NT, int TILE, int P>
__global__ void __launch_bounds__(NT) k_degrid_sep(const DegridArgs a, const int cls) {
  constexpr int R = sep_rows(SMIN, SMAX, NT);
  constexpr int NW = NT / 32;
  constexpr int B = 32 / (2 * P);
  using L = SepLayout<SMAX, TILE, P>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float2* s_f = reinterpret_cast<float2*>(smem + L::tile_bytes);
  float2* s_ph = reinterpret_cast<float2*>(smem + L::tile_bytes + L::f_bytes);    // [stage] (a_bytes >= this)
  long long* s_fxo = reinterpret_cast<long long*>(smem + L::tile_bytes + L::f_bytes + L::a_bytes);
  long long* s_fyo = s_fxo + kSepStage;
  int* s_pack = reinterpret_cast<int*>(s_fyo + kSepStage);
  int* s_src = s_pack + kSepStage;
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
    const int S = wi.S, U = TILE + S - 1;
    const int X0 = wi.tile_x * TILE, Y0 = wi.tile_y * TILE;
    const int G = NT / S;
    const bool active = tid < G * S;
    const int rx = tid % S, ry0 = tid / S;
    for (int i = tid; i < U * U; i += NT) {
      const int ly = i / U, lx = i - ly * U;
      const int gy = Y0 + ly, gx = X0 + lx;
      const bool in = gy < a.N && gx < a.N;
      const float2* src = reinterpret_cast<const float2*>(a.grid) + ((size_t)gy * a.N + gx) * P;
#pragma unroll
      for (int p = 0; p < P; ++p) tile[i * P + p] = in ? __ldg(src + p) : make_float2(0.f, 0.f);
    }
    for (int c0 = 0; c0 < wi.count; c0 += kSepStage) {
      const int nst = min(kSepStage, wi.count - c0);
      __syncthreads();
      if (tid < nst) {
        const SampleRec rc = a.rec[wi.start + c0 + tid];
        const long long base = a.sep_off[rc.cf];
        s_fxo[tid] = base + (long long)rc.ox * S;
        s_fyo[tid] = base + (long long)(a.OS + 1) * S + (long long)rc.oy * S;
        s_pack[tid] = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | ((rc.p0x % S) << 16) | ((rc.p0y % S) << 24);
        s_src[tid] = rc.src;
        float2 ph = make_float2(1.f, 0.f);
        if (a.has_phase) ph = sample_phasor(a.uvw, a.freq, a.C, rc.src, a.dl, a.dm, a.dn);
        s_ph[tid] = ph;
      }
      __syncthreads();
      for (int i = tid; i < nst * 2 * S; i += NT) {
        const int j = i / (2 * S), r = i - j * 2 * S;
        const long long src = r < S ? s_fxo[j] + r : s_fyo[j] + (r - S);
        s_f[(j * 2 + (r < S ? 0 : 1)) * SMAX + (r < S ? r : r - S)] =
            __ldg(reinterpret_cast<const float2*>(a.sep) + src);
      }
      __syncthreads();
      for (int j0 = 0; j0 < nst; j0 += B) {
        float vals[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) vals[q] = 0.f;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int j = j0 + b;
          if (active && j < nst) {
            const int pk = s_pack[j];
            const int dx = pk & 0xff, dy = (pk >> 8) & 0xff, mx = (pk >> 16) & 0xff, my = (pk >> 24) & 0xff;
            int tx = rx - mx;
            tx += (tx < 0) ? S : 0;
            const int X = dx + tx;
            int ty0 = ry0 - my;
            ty0 += (ty0 < 0) ? S : 0;
            const float2* fyrow = s_f + (j * 2 + 1) * SMAX;
            float2 part[P];
#pragma unroll
            for (int p = 0; p < P; ++p) part[p] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < R; ++k) {
              if (ry0 + k * G < S) {
                int ty = ty0 + k * G;
                ty -= (ty >= S) ? S : 0;
                const float2 f = fyrow[ty];
                const float2* g = tile + ((dy + ty) * U + X) * P;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                  const float2 gv = g[p];
                  part[p].x = fmaf(f.x, gv.x, fmaf(-f.y, gv.y, part[p].x));
                  part[p].y = fmaf(f.x, gv.y, fmaf(f.y, gv.x, part[p].y));
                }
              }
            }
            const float2 fxv = s_f[(j * 2) * SMAX + tx];
#pragma unroll
            for (int p = 0; p < P; ++p) {
              vals[b * 2 * P + 2 * p] = fxv.x * part[p].x - fxv.y * part[p].y;
              vals[b * 2 * P + 2 * p + 1] = fxv.x * part[p].y + fxv.y * part[p].x;
            }
          }
        }
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
            const float2 ph = s_ph[j];
            const float out = (comp & 1) ? (v * ph.x - partner * ph.y) : (v * ph.x + partner * ph.y);
            a.vis_out[(size_t)s_src[j] * 2 * P + comp] = out;
          }
        }
        buf ^= 1;
      }
    }
  }
}

template <int CLS, int P>
awg_status run_grid_sep(const GridArgs& a, int sms, cudaStream_t st) {
  constexpr ClassCfg cc = kClasses[CLS];
  constexpr int smin = CLS == 0 ? 0 : kClasses[CLS > 0 ? CLS - 1 : 0].smax;
  using L = SepLayout<cc.smax, cc.tile, P>;
  auto kern = k_grid_sep<smin, cc.smax, cc.nt, cc.tile, P>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cc.nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "separable gridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, cc.nt, L::bytes, st>>>(a, CLS);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

template <int CLS, int P>
awg_status run_degrid_sep(const DegridArgs& a, int sms, cudaStream_t st) {
  constexpr ClassCfg cc = kClasses[CLS];
  constexpr int smin = CLS == 0 ? 0 : kClasses[CLS > 0 ? CLS - 1 : 0].smax;
  using L = SepLayout<cc.smax, cc.tile, P>;
  auto kern = k_degrid_sep<smin, cc.smax, cc.nt, cc.tile, P>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cc.nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "separable degridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, cc.nt, L::bytes, st>>>(a, CLS);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

#define AWG_FOR_SEP_CLASSES_AND_POLS(M) \
  M(0, 1) M(0, 2) M(0, 4) M(1, 1) M(1, 2) M(1, 4) M(2, 1) M(2, 2) M(2, 4) M(3, 1) M(3, 2) M(3, 4) M(4, 1) M(4, 2) M(4, 4) \
  M(5, 1) M(5, 2) M(5, 4)

#define AWG_DECLARE_GRID_SEP(C, P) extern template awg_status run_grid_sep<C, P>(const GridArgs&, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_SEP(C, P) \
  extern template awg_status run_degrid_sep<C, P>(const DegridArgs&, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_SEP(C, P) template awg_status run_grid_sep<C, P>(const GridArgs&, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_SEP(C, P) \
  template awg_status run_degrid_sep<C, P>(const DegridArgs&, int, cudaStream_t);

}  // namespace awg
