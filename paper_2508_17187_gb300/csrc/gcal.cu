// Direction-independent G-Jones calibration (Sec. 5.1, Architectural View for Calibration):
//   k_vavg       Eq. VAvg - per solution interval of sol_int integrations x sol_chan channels,
//                parallel-hand product and baseline, the sums N = sum w V conj(M) and
//                D = sum w |M|^2 (X = N / D is the weighted average of V / M, and D its weight;
//                the iteration needs only w X = N and w = D).  One pass over the data, HBM-bound.
//   k_gain_solve Eq. CalUpdateDir / Eq. CalUpdateModel - the fixed-point iteration for the
//                antenna gains of one (solution interval, polarisation), with the exit test
//                max_i |g_i^{k+1} - g_i^k| < delta, then the phase of a reference antenna
//                removed (the solution is defined up to a common phase).
// The model visibilities come from degrid_visibilities (Eq. VMod).
//
// Precision: GB300's FP64 rate is 1/64 of its FP32 rate, so the data pass runs in FP32: every
// product rounded once, per-lane sums Kahan-compensated, a 5-level FP32 tree across the lanes
// (relative error of N and D within ~10 u of sum w |V| |M|, u = 2^-24, whatever the interval
// length).  The iteration is FP64.
#include <cuda_runtime.h>

#include "awg_internal.h"

namespace awg {
namespace {

struct GcalDims {
  int64_t n_rows;
  int C, P, n_bl, n_ant, n_pp, sol_int, sol_chan, n_ts, n_fs, n_int;
  int pol[2];   // the parallel-hand products among the P pols
};

// The parallel hands of one (row, channel) sample: whole-sample vector loads (the P pols of a
// sample are contiguous), so every fetched sector is used.
template <int P>
__device__ __forceinline__ void load_hands(const float2* __restrict__ v, const float* __restrict__ w, int64_t s,
                                           float2 (&vh)[2], float (&wh)[2]) {
  if constexpr (P == 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(v + s * 4));
    const float4 b = __ldg(reinterpret_cast<const float4*>(v + s * 4) + 1);
    const float4 ww = __ldg(reinterpret_cast<const float4*>(w + s * 4));
    vh[0] = make_float2(a.x, a.y);
    vh[1] = make_float2(b.z, b.w);
    wh[0] = ww.x;
    wh[1] = ww.w;
  } else if constexpr (P == 2) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(v + s * 2));
    const float2 ww = __ldg(reinterpret_cast<const float2*>(w + s * 2));
    vh[0] = make_float2(a.x, a.y);
    vh[1] = make_float2(a.z, a.w);
    wh[0] = ww.x;
    wh[1] = ww.y;
  } else {
    vh[0] = __ldg(v + s);
    wh[0] = __ldg(w + s);
    vh[1] = make_float2(0.f, 0.f);
    wh[1] = 0.f;
  }
}

// Kahan-compensated FP32 accumulation: sum + c carries the running total.
struct KSum {
  float sum = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = sum + y;
    c = (t - sum) - y;
    sum = t;
  }
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// One CTA per solution cell (time interval, channel block); its warps take baselines, the lanes
// of a warp take the (integration, channel) samples of one baseline.  Output per (cell, hand,
// baseline): float4 (Re N, Im N, D, 0).
template <int P>
__global__ void __launch_bounds__(256) k_vavg(GcalDims d, const float2* __restrict__ vis, const float2* __restrict__ mod,
                                              const float* __restrict__ weight, float4* __restrict__ ND) {
  constexpr int H = P == 1 ? 1 : 2;
  const int ts = blockIdx.x / d.n_fs, fs = blockIdx.x - (blockIdx.x / d.n_fs) * d.n_fs;
  const int t0 = ts * d.sol_int, t1 = min(t0 + d.sol_int, d.n_int);
  const int c0 = fs * d.sol_chan, c1 = min(c0 + d.sol_chan, d.C);
  const int nc = c1 - c0, ns = (t1 - t0) * nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = warp; b < d.n_bl; b += nw) {
    KSum nr[2], ni[2], den[2];
#pragma unroll 4
    for (int k = lane; k < ns; k += 32) {
      const int t = t0 + k / nc, c = c0 + k % nc;
      const int64_t s = ((int64_t)t * d.n_bl + b) * d.C + c;
      float2 v[2], m[2];
      float w[2], wm[2];
      load_hands<P>(vis, weight, s, v, w);
      load_hands<P>(mod, weight, s, m, wm);
#pragma unroll
      for (int q = 0; q < H; ++q) {
        if (!(w[q] > 0.f)) continue;
        // w V conj(M) and w |M|^2
        const float re = fmaf(v[q].x, m[q].x, v[q].y * m[q].y);
        const float im = fmaf(v[q].y, m[q].x, -(v[q].x * m[q].y));
        const float mm = fmaf(m[q].x, m[q].x, m[q].y * m[q].y);
        nr[q].add(w[q] * re);
        ni[q].add(w[q] * im);
        den[q].add(w[q] * mm);
      }
    }
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const float a = warp_sum(nr[q].sum - nr[q].c);
      const float bb = warp_sum(ni[q].sum - ni[q].c);
      const float cc = warp_sum(den[q].sum - den[q].c);
      if (lane == 0) ND[(((int64_t)ts * d.n_fs + fs) * H + q) * d.n_bl + b] = make_float4(a, bb, cc, 0.f);
    }
  }
}

constexpr int kMaxAnt = 128;
constexpr int kMaxBl = kMaxAnt * (kMaxAnt - 1) / 2;

// Dynamic shared memory of k_gain_solve: the solution's N (2 values) and D per baseline as FP32,
// then as T again when T = double (the FP64 phase reads that copy; with T = float it converts the
// FP32 one), then for every antenna its neighbour entries (b << 8) | (j << 1) | (1 if the antenna
// is ant2 of b, so that w_ij X_ij = conj(N_b)), [n_ant][n_ant - 1].
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <typename T>
size_t gain_solve_smem(int n_bl, int n_ant) {
  const size_t nd32 = align16((size_t)n_bl * 3 * sizeof(float));
  const size_t nd64 = sizeof(T) == sizeof(double) ? align16((size_t)n_bl * 3 * sizeof(double)) : 0;
  return nd32 + nd64 + sizeof(int) * (size_t)n_ant * (n_ant - 1);
}

// One update of antenna i (Eq. CalUpdateDir, then Eq. CalUpdateModel) in precision R:
//   g_i' = sum_j g_j w_ij X_ij / sum_j |g_j|^2 w_ij,  w_ij X_ij = N_b or conj(N_b), w_ij = D_b,
//   g_i <- (1 - alpha) g_i + alpha g_i'.
// Returns the new gain in (re, im) and |change|^2.  (The FP64 phase is bound by the FP64 pipe's
// throughput: one thread per antenna keeps every FP64 operation useful.)
template <typename R, typename S>
__device__ __forceinline__ R gain_update(int deg, const int* __restrict__ adj, const S* __restrict__ nd,
                                         const R* __restrict__ gre, const R* __restrict__ gim,
                                         const R* __restrict__ gg, R alpha, int i, R& re, R& im) {
  R num_r = R(0), num_i = R(0), den = R(0);
  for (int k = 0; k < deg; ++k) {
    const int e = adj[k], b = e >> 8, j = (e >> 1) & 127;
    const R nr = (R)nd[3 * b];
    const R ni = (e & 1) ? -(R)nd[3 * b + 1] : (R)nd[3 * b + 1];
    const R gx = gre[j], gy = gim[j];
    num_r = fma(gx, nr, fma(-gy, ni, num_r));
    num_i = fma(gx, ni, fma(gy, nr, num_i));
    den = fma(gg[j], (R)nd[3 * b + 2], den);
  }
  const R gx = gre[i], gy = gim[i];
  re = gx;
  im = gy;
  if (den > R(0)) {
    const R r = alpha / den;
    re = fma(r, num_r, (R(1) - alpha) * gx);
    im = fma(r, num_i, (R(1) - alpha) * gy);
  }
  const R dx = re - gx, dy = im - gy;
  return dx * dx + dy * dy;
}

// Largest of v over the CTA's threads (all threads call it; s_red holds one value per warp).
template <typename R>
__device__ __forceinline__ R block_max(R v, R* s_red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
  __syncthreads();
  R m = R(0);
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, s_red[k]);
  return m;
}

// Relative change below which the FP32 phase hands over to FP64: 3e-5 of the largest gain is
// ~500 u (u = 2^-24), far above the rounding of an FP32 update.  Below kStall32 the FP32 phase also
// hands over as soon as the largest change stops shrinking (where its rounding would take over),
// so it cannot stall; above it a non-monotone early step does not end the phase.
constexpr float kTau32 = 3e-5f;
constexpr float kStall32 = 1e-4f;

// One CTA per (interval, hand): thread i owns antenna i; Jacobi order (every g_j of the previous
// iteration).  The iteration runs in FP32 while the largest change is above kTau32 max |g| (the
// FP64 pipe of GB300 is 1/64 of the FP32 one), then in FP64 until max_i |change| < delta.  A delta
// coarser than kTau32 max |g| is tested in the FP32 phase.
template <typename T>
__global__ void __launch_bounds__(kMaxAnt) k_gain_solve(GcalDims d, const int32_t* __restrict__ ant1,
                                                         const int32_t* __restrict__ ant2,
                                                         const float4* __restrict__ ND, double alpha, double delta,
                                                         int max_iter, int ref_ant, double2* __restrict__ gains,
                                                         int32_t* __restrict__ iters) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  float* s_nd32 = reinterpret_cast<float*>(s_raw);   // [n_bl][3]
  const size_t o64 = align16((size_t)d.n_bl * 3 * sizeof(float));
  T* s_nd = sizeof(T) == sizeof(double) ? reinterpret_cast<T*>(s_raw + o64) : reinterpret_cast<T*>(s_nd32);
  const size_t oadj = o64 + (sizeof(T) == sizeof(double) ? align16((size_t)d.n_bl * 3 * sizeof(double)) : 0);
  int* s_adj = reinterpret_cast<int*>(s_raw + oadj);
  __shared__ float g32r[kMaxAnt], g32i[kMaxAnt], gg32[kMaxAnt];
  __shared__ double gre[kMaxAnt], gim[kMaxAnt], gg[kMaxAnt];
  __shared__ float s_red32[kMaxAnt / 32];
  __shared__ double s_red[kMaxAnt / 32];
  const int sol = blockIdx.x;   // (ts, fs, q)
  const float4* nd = ND + (int64_t)sol * d.n_bl;
  const int i = threadIdx.x;
  for (int b = i; b < d.n_bl; b += blockDim.x) {
    const float4 v = nd[b];
    s_nd32[3 * b] = v.x;
    s_nd32[3 * b + 1] = v.y;
    s_nd32[3 * b + 2] = v.z;
    if (sizeof(T) == sizeof(double)) {
      s_nd[3 * b] = (T)v.x;
      s_nd[3 * b + 1] = (T)v.y;
      s_nd[3 * b + 2] = (T)v.z;
    }
  }
  const int deg_max = d.n_ant - 1;
  int* adj = s_adj + i * deg_max;
  int deg = 0;
  const bool own = i < d.n_ant;
  if (own) {
    g32r[i] = 1.f;
    g32i[i] = 0.f;
    gg32[i] = 1.f;
    for (int b = 0; b < d.n_bl && deg < deg_max; ++b) {
      const int a = ant1[b], c = ant2[b];
      if (a < 0 || c < 0 || a >= d.n_ant || c >= d.n_ant || a == c) continue;
      if (a == i) adj[deg++] = (b << 8) | (c << 1);
      else if (c == i) adj[deg++] = (b << 8) | (a << 1) | 1;
    }
  }
  const double delta2 = delta * delta;
  __syncthreads();
  int it = 0;
  bool done = false;
  float m_prev = INFINITY;
  // FP32 phase
  while (it < max_iter) {
    float re = 0.f, im = 0.f, c2 = 0.f;
    if (own) c2 = gain_update<float, float>(deg, adj, s_nd32, g32r, g32i, gg32, (float)alpha, i, re, im);
    const float m = block_max(c2, s_red32);
    __syncthreads();   // every thread has read s_red32 and the old gains
    const float gm = block_max(own ? re * re + im * im : 0.f, s_red32);
    if (own) {
      g32r[i] = re;
      g32i[i] = im;
      gg32[i] = re * re + im * im;
    }
    ++it;
    __syncthreads();
    const double switch2 = (double)(kTau32 * kTau32) * (double)gm;
    const double stall2 = (double)(kStall32 * kStall32) * (double)gm;
    if ((double)m < switch2 || ((double)m < stall2 && !(m < m_prev))) {
      done = delta2 >= switch2 && (double)m < delta2;
      break;
    }
    m_prev = m;
  }
  // FP64 phase
  if (own) {
    gre[i] = g32r[i];
    gim[i] = g32i[i];
    gg[i] = (double)g32r[i] * g32r[i] + (double)g32i[i] * g32i[i];
  }
  __syncthreads();
  while (!done && it < max_iter) {
    double re = 0.0, im = 0.0, c2 = 0.0;
    if (own) c2 = gain_update<double, T>(deg, adj, s_nd, gre, gim, gg, alpha, i, re, im);
    const double m = block_max(c2, s_red);
    __syncthreads();
    if (own) {
      gre[i] = re;
      gim[i] = im;
      gg[i] = re * re + im * im;
    }
    ++it;
    __syncthreads();
    done = m < delta2 || (m == 0.0 && delta > 0.0);
  }
  if (own) {
    // remove the reference antenna's phase: g_i conj(g_ref) / |g_ref|
    const double rx = gre[ref_ant], ry = gim[ref_ant];
    const double ar = hypot(rx, ry);
    double ox = gre[i], oy = gim[i];
    if (ar > 0.0) {
      const double tx = (ox * rx + oy * ry) / ar;
      oy = (oy * rx - ox * ry) / ar;
      ox = tx;
    }
    gains[(int64_t)sol * d.n_ant + i] = make_double2(ox, oy);
  }
  if (threadIdx.x == 0) iters[sol] = it;
}

awg_status gcal_dims(int64_t n_rows, int32_t n_chan, int32_t n_pol, int32_t n_bl, int32_t n_ant, int32_t sol_int,
                     int32_t sol_chan, GcalDims& d) {
  if (n_rows < 1 || n_chan < 1 || n_bl < 1 || n_ant < 2) return set_error(AWG_ERR_INVALID_ARG, "empty calibration problem");
  if (n_pol != 1 && n_pol != 2 && n_pol != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  if (n_ant > kMaxAnt || n_bl > kMaxBl) return set_error(AWG_ERR_UNSUPPORTED, "more than 128 antennas");
  if (n_rows % n_bl != 0) return set_error(AWG_ERR_INVALID_ARG, "n_rows must be a multiple of n_bl (time-major rows)");
  if (sol_int < 1 || sol_chan < 1) return set_error(AWG_ERR_INVALID_ARG, "solution intervals must be >= 1");
  d.n_rows = n_rows;
  d.C = n_chan;
  d.P = n_pol;
  d.n_bl = n_bl;
  d.n_ant = n_ant;
  d.n_pp = n_pol == 1 ? 1 : 2;
  d.pol[0] = 0;
  d.pol[1] = n_pol == 4 ? 3 : 1;
  d.sol_int = sol_int;
  d.sol_chan = sol_chan;
  d.n_int = (int)(n_rows / n_bl);
  d.n_ts = (d.n_int + sol_int - 1) / sol_int;
  d.n_fs = (n_chan + sol_chan - 1) / sol_chan;
  return AWG_OK;
}

}  // namespace
}  // namespace awg

using namespace awg;

extern "C" int64_t gcal_workspace_bytes(int64_t n_rows, int32_t n_chan, int32_t n_pol, int32_t n_bl, int32_t sol_int,
                                        int32_t sol_chan) {
  if (n_bl < 1 || sol_int < 1 || sol_chan < 1 || n_chan < 1 || n_rows < 1) return 0;
  const int64_t n_int = n_rows / n_bl;
  const int64_t n_sol = ((n_int + sol_int - 1) / sol_int) * ((n_chan + sol_chan - 1) / sol_chan) * (n_pol == 1 ? 1 : 2);
  return n_sol * n_bl * (int64_t)sizeof(float4);
}

extern "C" awg_status gcal_solve(const void* vis, const void* model, const float* weight, int64_t n_rows, int32_t n_chan,
                                 int32_t n_pol, int32_t n_bl, const int32_t* ant1, const int32_t* ant2, int32_t n_ant,
                                 int32_t sol_int, int32_t sol_chan, double alpha, double delta, int32_t max_iter,
                                 int32_t ref_ant, void* gains, int32_t* iterations, void* workspace, void* stream) {
  NvtxRange nvtx_range("awg gcal_solve");
  GcalDims d;
  awg_status s = gcal_dims(n_rows, n_chan, n_pol, n_bl, n_ant, sol_int, sol_chan, d);
  if (s != AWG_OK) return s;
  if (!vis || !model || !weight || !ant1 || !ant2 || !gains || !iterations || !workspace)
    return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  if (!(alpha > 0.0 && alpha <= 1.0)) return set_error(AWG_ERR_INVALID_ARG, "alpha must be in (0, 1]");
  if (!(delta >= 0.0) || max_iter < 1) return set_error(AWG_ERR_INVALID_ARG, "delta >= 0 and max_iter >= 1 required");
  if (ref_ant < 0 || ref_ant >= n_ant) return set_error(AWG_ERR_INVALID_ARG, "ref_ant out of range");
  if (((uintptr_t)workspace & 15) != 0) return set_error(AWG_ERR_INVALID_ARG, "workspace must be 16-byte aligned");
  const int64_t n_sol = (int64_t)d.n_ts * d.n_fs * d.n_pp;
  float4* ND = (float4*)workspace;
  cudaStream_t st = (cudaStream_t)stream;
  if (((uintptr_t)vis | (uintptr_t)model | (uintptr_t)weight) & 15)
    return set_error(AWG_ERR_INVALID_ARG, "vis, model and weight must be 16-byte aligned");
  auto kv = n_pol == 4 ? k_vavg<4> : n_pol == 2 ? k_vavg<2> : k_vavg<1>;
  kv<<<d.n_ts * d.n_fs, 256, 0, st>>>(d, (const float2*)vis, (const float2*)model, weight, ND);
  AWG_CUDA_TRY(cudaGetLastError());
  const int threads = ((n_ant + 31) / 32) * 32;
  // N and D staged as FP64 when that fits next to the neighbour lists, else as FP32
  constexpr size_t kSmemMax = 200 * 1024;
  const bool dbl = gain_solve_smem<double>(n_bl, n_ant) <= kSmemMax;
  const size_t smem = dbl ? gain_solve_smem<double>(n_bl, n_ant) : gain_solve_smem<float>(n_bl, n_ant);
  static bool attr_set = false;
  if (!attr_set) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(k_gain_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    AWG_CUDA_TRY(cudaFuncSetAttribute(k_gain_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
    attr_set = true;
  }
  if (dbl)
    k_gain_solve<double><<<(int)n_sol, threads, smem, st>>>(d, ant1, ant2, ND, alpha, delta, max_iter, ref_ant,
                                                            (double2*)gains, iterations);
  else
    k_gain_solve<float><<<(int)n_sol, threads, smem, st>>>(d, ant1, ant2, ND, alpha, delta, max_iter, ref_ant,
                                                           (double2*)gains, iterations);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(2);
  return AWG_OK;
}
