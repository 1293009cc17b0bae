// Direction-independent G-Jones calibration (Sec. 5.1, Architectural View for Calibration):
//   k_vavg       Eq. VAvg - the model-normalised visibilities of every baseline averaged over a
//                solution interval of sol_int integrations x sol_chan channels, per parallel-hand
//                polarisation product: X = sum w V conj(M) / sum w |M|^2 with weight sum w |M|^2
//                (one pass over the data, HBM-bound);
//   k_gain_solve Eq. CalUpdateDir / Eq. CalUpdateModel - the fixed-point iteration for the
//                antenna gains of one (solution interval, polarisation), with the exit test
//                max_i |g_i^{k+1} - g_i^k| < delta, then the phase of a reference antenna
//                removed (the solution is defined up to a common phase).
// The model visibilities come from degrid_visibilities (Eq. VMod).  Sums and the iteration are
// FP64.
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

// One CTA per solution cell (time interval, channel block); its warps take baselines, the lanes
// of a warp take the (integration, channel) samples of one baseline.
template <int P>
__global__ void __launch_bounds__(256) k_vavg(GcalDims d, const float2* __restrict__ vis, const float2* __restrict__ mod,
                                              const float* __restrict__ weight, double2* __restrict__ X,
                                              double* __restrict__ Wt) {
  constexpr int H = P == 1 ? 1 : 2;
  const int ts = blockIdx.x / d.n_fs, fs = blockIdx.x - (blockIdx.x / d.n_fs) * d.n_fs;
  const int t0 = ts * d.sol_int, t1 = min(t0 + d.sol_int, d.n_int);
  const int c0 = fs * d.sol_chan, c1 = min(c0 + d.sol_chan, d.C);
  const int nc = c1 - c0, ns = (t1 - t0) * nc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = warp; b < d.n_bl; b += nw) {
    double nr[2] = {0.0, 0.0}, ni[2] = {0.0, 0.0}, den[2] = {0.0, 0.0};
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
        nr[q] += (double)w[q] * ((double)v[q].x * m[q].x + (double)v[q].y * m[q].y);
        ni[q] += (double)w[q] * ((double)v[q].y * m[q].x - (double)v[q].x * m[q].y);
        den[q] += (double)w[q] * ((double)m[q].x * m[q].x + (double)m[q].y * m[q].y);
      }
    }
#pragma unroll
    for (int q = 0; q < H; ++q) {
      for (int o = 16; o > 0; o >>= 1) {
        nr[q] += __shfl_xor_sync(0xffffffffu, nr[q], o);
        ni[q] += __shfl_xor_sync(0xffffffffu, ni[q], o);
        den[q] += __shfl_xor_sync(0xffffffffu, den[q], o);
      }
      if (lane == 0) {
        const int64_t o = (((int64_t)ts * d.n_fs + fs) * H + q) * d.n_bl + b;
        X[o] = den[q] > 0.0 ? make_double2(nr[q] / den[q], ni[q] / den[q]) : make_double2(0.0, 0.0);
        Wt[o] = den[q];
      }
    }
  }
}

constexpr int kMaxAnt = 128;
constexpr int kMaxBl = kMaxAnt * (kMaxAnt - 1) / 2;

// Dynamic shared memory: for every antenna its baselines, as (b << 1) | (1 if the antenna is
// ant2 of b, so X_ij = conj(X_b)), [n_ant][n_ant - 1], then the counts [n_ant].
__global__ void __launch_bounds__(kMaxAnt) k_gain_solve(GcalDims d, const int32_t* __restrict__ ant1,
                                                         const int32_t* __restrict__ ant2,
                                                         const double2* __restrict__ X, const double* __restrict__ Wt,
                                                         double alpha, double delta, int max_iter, int ref_ant,
                                                         double2* __restrict__ gains, int32_t* __restrict__ iters) {
  extern __shared__ int s_adj[];
  __shared__ double2 g[kMaxAnt];
  __shared__ double s_red[kMaxAnt / 32];
  __shared__ int s_done;
  const int sol = blockIdx.x;   // (ts, fs, q)
  const double2* x = X + (int64_t)sol * d.n_bl;
  const double* w = Wt + (int64_t)sol * d.n_bl;
  const int i = threadIdx.x;
  const int deg_max = d.n_ant - 1;
  int* adj = s_adj + i * deg_max;
  int deg = 0;
  if (i < d.n_ant) {
    g[i] = make_double2(1.0, 0.0);
    for (int b = 0; b < d.n_bl && deg < deg_max; ++b) {
      const int a = ant1[b], c = ant2[b];
      if (a < 0 || c < 0 || a >= d.n_ant || c >= d.n_ant || a == c) continue;
      if (a == i) adj[deg++] = b << 1;
      else if (c == i) adj[deg++] = (b << 1) | 1;
    }
  }
  if (i == 0) s_done = 0;
  __syncthreads();
  int it = 0;
  for (; it < max_iter; ++it) {
    double2 gn = make_double2(0.0, 0.0);
    double change = 0.0;
    if (i < d.n_ant) {
      // Eq. CalUpdateDir: sum over j != i of g_j X_ij w_ij / sum |g_j|^2 w_ij; X_ij = conj(X_ji)
      double num_r = 0.0, num_i = 0.0, den = 0.0;
      for (int k = 0; k < deg; ++k) {
        const int e = adj[k], b = e >> 1;
        const int j = (e & 1) ? ant1[b] : ant2[b];
        const double2 xb = x[b];
        const double xi = (e & 1) ? -xb.y : xb.y;
        const double2 gj = g[j];
        const double wb = w[b];
        num_r += wb * (gj.x * xb.x - gj.y * xi);
        num_i += wb * (gj.x * xi + gj.y * xb.x);
        den += wb * (gj.x * gj.x + gj.y * gj.y);
      }
      const double2 gi = g[i];
      if (den > 0.0) {   // Eq. CalUpdateModel
        gn = make_double2((1.0 - alpha) * gi.x + alpha * num_r / den, (1.0 - alpha) * gi.y + alpha * num_i / den);
      } else {
        gn = gi;
      }
      change = hypot(gn.x - gi.x, gn.y - gi.y);
    }
    // largest change over the antennas
    for (int o = 16; o > 0; o >>= 1) change = fmax(change, __shfl_xor_sync(0xffffffffu, change, o));
    if ((i & 31) == 0) s_red[i >> 5] = change;
    __syncthreads();
    if (i < d.n_ant) g[i] = gn;
    if (i == 0) {
      double m = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, s_red[k]);
      s_done = m < delta;
    }
    __syncthreads();
    if (s_done) {
      ++it;
      break;
    }
  }
  if (i < d.n_ant) {
    // remove the reference antenna's phase: g_i conj(g_ref) / |g_ref|
    const double2 gr = g[ref_ant];
    const double ar = hypot(gr.x, gr.y);
    double2 o = g[i];
    if (ar > 0.0) o = make_double2((o.x * gr.x + o.y * gr.y) / ar, (o.y * gr.x - o.x * gr.y) / ar);
    gains[(int64_t)sol * d.n_ant + i] = o;
  }
  if (i == 0) iters[sol] = it;
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
  return n_sol * n_bl * (int64_t)(sizeof(double2) + sizeof(double));
}

extern "C" awg_status gcal_solve(const void* vis, const void* model, const float* weight, int64_t n_rows, int32_t n_chan,
                                 int32_t n_pol, int32_t n_bl, const int32_t* ant1, const int32_t* ant2, int32_t n_ant,
                                 int32_t sol_int, int32_t sol_chan, double alpha, double delta, int32_t max_iter,
                                 int32_t ref_ant, void* gains, int32_t* iterations, void* workspace, void* stream) {
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
  double2* X = (double2*)workspace;
  double* Wt = (double*)(X + n_sol * d.n_bl);
  cudaStream_t st = (cudaStream_t)stream;
  if (((uintptr_t)vis | (uintptr_t)model | (uintptr_t)weight) & 15)
    return set_error(AWG_ERR_INVALID_ARG, "vis, model and weight must be 16-byte aligned");
  auto kv = n_pol == 4 ? k_vavg<4> : n_pol == 2 ? k_vavg<2> : k_vavg<1>;
  kv<<<d.n_ts * d.n_fs, 256, 0, st>>>(d, (const float2*)vis, (const float2*)model, weight, X, Wt);
  AWG_CUDA_TRY(cudaGetLastError());
  const int threads = ((n_ant + 31) / 32) * 32;
  const size_t adj_bytes = sizeof(int) * (size_t)n_ant * (n_ant - 1);
  static bool attr_set = false;
  if (!attr_set) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(k_gain_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(int) * kMaxAnt * (kMaxAnt - 1))));
    attr_set = true;
  }
  k_gain_solve<<<(int)n_sol, threads, adj_bytes, st>>>(d, ant1, ant2, X, Wt, alpha, delta, max_iter, ref_ant,
                                                       (double2*)gains, iterations);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(2);
  return AWG_OK;
}
