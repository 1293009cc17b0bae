// Plain FP64 baseline of gridding and degridding: one launch per channel, one thread per row, no
// sorting, no tiling, every tap an FP64 multiply-add (gridding: an FP64 atomic into a complex128
// grid).  This is the straightforward GPU port of the operators (Eq. IMAGE-MOD,
// Eq. ME-MOD-GRIDDED) that the batched FP32 kernels are measured against; it uses the same index
// rules and the CF set's full FP32 tables, widened to FP64.
#include <cuda_runtime.h>

#include "awg_internal.h"

namespace awg {
namespace {

struct PlainArgs {
  const double* uvw;
  double sc;          // nu / c of this channel
  int chan, C, N, OS, use_w, n_w, n_pa, n_sb, n_signed, sb, P;
  double inv_dw, scale, half;
  const int32_t* pa_bin;
  const int32_t* sup;
  const int64_t* cf_off;
  const float2* cf;
  int64_t R;
};

// The index rules of plan.cu for one sample; returns false for a dropped sample.
__device__ bool plain_index(const PlainArgs& a, int64_t r, int* cf, int* S, int* p0x, int* p0y, int* ox, int* oy) {
  const double u = __dmul_rn(a.uvw[3 * r], a.sc);
  const double v = __dmul_rn(a.uvw[3 * r + 1], a.sc);
  const double w = __dmul_rn(a.uvw[3 * r + 2], a.sc);
  const double x = __dadd_rn(__dmul_rn(u, a.scale), a.half);
  const double y = __dadd_rn(__dmul_rn(v, a.scale), a.half);
  if (!isfinite(x) || !isfinite(y)) return false;
  int ks = 0;
  if (a.use_w) {
    const double k = floor(__dadd_rn(__dmul_rn(fabs(w), a.inv_dw), 0.5));
    if (!(k <= (double)(a.n_w - 1))) return false;
    ks = a.n_w - 1 + (w < 0.0 ? -(int)k : (int)k);
  }
  int pa = 0;
  if (a.n_pa > 1) {
    pa = a.pa_bin[r];
    if (pa < 0 || pa >= a.n_pa) return false;
  }
  *cf = (pa * a.n_sb + a.sb) * a.n_signed + ks;
  *S = a.sup[*cf];
  const double hS = 0.5 * (double)*S;
  const double hx = __dsub_rn(x, hS), hy = __dsub_rn(y, hS);
  const double lim = (double)(a.N - *S);
  if (!((hx >= -1.0) && (hx < lim) && (hy >= -1.0) && (hy < lim))) return false;
  const double px = __dadd_rn(floor(hx), 1.0), py = __dadd_rn(floor(hy), 1.0);
  *ox = (int)floor(__dadd_rn(__dmul_rn(__dsub_rn(px, hx), (double)a.OS), 0.5));
  *oy = (int)floor(__dadd_rn(__dmul_rn(__dsub_rn(py, hy), (double)a.OS), 0.5));
  *p0x = (int)px;
  *p0y = (int)py;
  return true;
}

__global__ void k_plain_grid(PlainArgs a, const float2* __restrict__ vis, const float* __restrict__ wt,
                             double* __restrict__ grid, double* __restrict__ sumwt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  int cf, S, p0x, p0y, ox, oy;
  if (!plain_index(a, r, &cf, &S, &p0x, &p0y, &ox, &oy)) return;
  const int64_t s = r * a.C + a.chan;
  double ar[4], ai[4];
  for (int p = 0; p < a.P; ++p) {
    const double wv = (double)wt[s * a.P + p];
    const float2 v = vis[s * a.P + p];
    ar[p] = wv * (double)v.x;
    ai[p] = wv * (double)v.y;
    atomicAdd(sumwt + p, wv);
  }
  const float2* tab = a.cf + a.cf_off[cf] + ((int64_t)oy * (a.OS + 1) + ox) * S * S;
  for (int ty = 0; ty < S; ++ty)
    for (int tx = 0; tx < S; ++tx) {
      const float2 c = tab[ty * S + tx];
      const double cr = (double)c.x, ci = -(double)c.y;   // conj(c)
      double* g = grid + (((int64_t)(p0y + ty) * a.N + p0x + tx) * a.P) * 2;
      for (int p = 0; p < a.P; ++p) {
        atomicAdd(g + 2 * p, cr * ar[p] - ci * ai[p]);
        atomicAdd(g + 2 * p + 1, cr * ai[p] + ci * ar[p]);
      }
    }
}

__global__ void k_plain_degrid(PlainArgs a, const double* __restrict__ grid, float2* __restrict__ vis_out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.R) return;
  const int64_t s = r * a.C + a.chan;
  int cf, S, p0x, p0y, ox, oy;
  double accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};
  if (plain_index(a, r, &cf, &S, &p0x, &p0y, &ox, &oy)) {
    const float2* tab = a.cf + a.cf_off[cf] + ((int64_t)oy * (a.OS + 1) + ox) * S * S;
    for (int ty = 0; ty < S; ++ty)
      for (int tx = 0; tx < S; ++tx) {
        const float2 c = tab[ty * S + tx];
        const double* g = grid + (((int64_t)(p0y + ty) * a.N + p0x + tx) * a.P) * 2;
        for (int p = 0; p < a.P; ++p) {
          accr[p] += (double)c.x * g[2 * p] - (double)c.y * g[2 * p + 1];
          acci[p] += (double)c.x * g[2 * p + 1] + (double)c.y * g[2 * p];
        }
      }
  }
  for (int p = 0; p < a.P; ++p) vis_out[s * a.P + p] = make_float2((float)accr[p], (float)acci[p]);
}

PlainArgs plain_args(CfSetImpl* cf, const double* uvw, int64_t R, int C, const int32_t* pa_bin, int P) {
  PlainArgs a;
  a.uvw = uvw;
  a.C = C;
  a.N = cf->p.grid_n;
  a.OS = cf->p.oversampling;
  a.use_w = cf->p.use_w;
  a.n_w = cf->p.use_w ? cf->p.n_wplanes : 1;
  a.n_pa = cf->p.n_pa_bins;
  a.n_sb = cf->p.n_subbands;
  a.n_signed = cf->n_signed;
  a.P = P;
  a.inv_dw = cf->p.use_w ? (double)(cf->p.n_wplanes - 1) / cf->p.w_max_lambda : 0.0;
  a.scale = (double)cf->p.grid_n * cf->p.cell_rad;
  a.half = (double)(cf->p.grid_n / 2);
  a.pa_bin = pa_bin;
  a.sup = cf->d_sup;
  a.cf_off = cf->d_off;
  a.cf = (const float2*)cf->d_data;
  a.R = R;
  return a;
}

awg_status plain_checks(CfSetImpl* cf, int64_t n_rows, int n_chan, const int32_t* pa_bin, const int32_t* chan_sb,
                        const double* freq_host, int P) {
  if (cf->separable || cf->p.cf_dtype != AWG_CF_FP32)
    return set_error(AWG_ERR_UNSUPPORTED, "the plain FP64 baseline needs a CF set with full FP32 tables");
  if (P != 1 && P != 2 && P != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  if (n_rows < 0 || n_chan < 1 || !freq_host) return set_error(AWG_ERR_INVALID_ARG, "bad rows / channels / freq");
  if (cf->p.n_pa_bins > 1 && !pa_bin) return set_error(AWG_ERR_INVALID_ARG, "pa_bin is required");
  if (cf->p.n_subbands > 1 && !chan_sb) return set_error(AWG_ERR_INVALID_ARG, "chan_subband (host) is required");
  return AWG_OK;
}

}  // namespace
}  // namespace awg

using namespace awg;

extern "C" awg_status grid_visibilities_plain_fp64(awg_cf_set hc, const double* uvw_m, int64_t n_rows,
                                                   const double* freq_hz_host, int32_t n_chan, int32_t chan_begin,
                                                   int32_t chan_end, const int32_t* pa_bin,
                                                   const int32_t* chan_subband_host, const void* vis,
                                                   const float* weight, int32_t n_pol, void* grid64,
                                                   double* sumwt, void* stream) {
  if (!hc || !uvw_m || !vis || !weight || !grid64 || !sumwt) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)hc;
  awg_status s = plain_checks(cf, n_rows, n_chan, pa_bin, chan_subband_host, freq_hz_host, n_pol);
  if (s != AWG_OK) return s;
  if (chan_begin < 0 || chan_end > n_chan || chan_begin > chan_end)
    return set_error(AWG_ERR_INVALID_ARG, "channel range out of bounds");
  cudaStream_t st = (cudaStream_t)stream;
  PlainArgs a = plain_args(cf, uvw_m, n_rows, n_chan, pa_bin, n_pol);
  for (int c = chan_begin; c < chan_end; ++c) {
    a.chan = c;
    a.sc = freq_hz_host[c] / kCLight;
    a.sb = cf->p.n_subbands > 1 ? chan_subband_host[c] : 0;
    if (n_rows == 0) continue;
    k_plain_grid<<<(unsigned)((n_rows + 127) / 128), 128, 0, st>>>(a, (const float2*)vis, weight, (double*)grid64,
                                                                    sumwt);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  return AWG_OK;
}

extern "C" awg_status degrid_visibilities_plain_fp64(awg_cf_set hc, const double* uvw_m, int64_t n_rows,
                                                     const double* freq_hz_host, int32_t n_chan, int32_t chan_begin,
                                                     int32_t chan_end, const int32_t* pa_bin,
                                                     const int32_t* chan_subband_host, const void* grid64,
                                                     void* vis_out, int32_t n_pol, void* stream) {
  if (!hc || !uvw_m || !grid64 || !vis_out) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)hc;
  awg_status s = plain_checks(cf, n_rows, n_chan, pa_bin, chan_subband_host, freq_hz_host, n_pol);
  if (s != AWG_OK) return s;
  if (chan_begin < 0 || chan_end > n_chan || chan_begin > chan_end)
    return set_error(AWG_ERR_INVALID_ARG, "channel range out of bounds");
  cudaStream_t st = (cudaStream_t)stream;
  PlainArgs a = plain_args(cf, uvw_m, n_rows, n_chan, pa_bin, n_pol);
  for (int c = chan_begin; c < chan_end; ++c) {
    a.chan = c;
    a.sc = freq_hz_host[c] / kCLight;
    a.sb = cf->p.n_subbands > 1 ? chan_subband_host[c] : 0;
    if (n_rows == 0) continue;
    k_plain_degrid<<<(unsigned)((n_rows + 127) / 128), 128, 0, st>>>(a, (const double*)grid64, (float2*)vis_out);
    AWG_CUDA_TRY(cudaGetLastError());
    count_launches(1);
  }
  return AWG_OK;
}
