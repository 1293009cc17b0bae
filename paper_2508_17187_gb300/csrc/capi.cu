// C ABI entry points of awgrid: argument checks, object lifetimes, CF-set upload.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "awg_internal.h"

namespace awg {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

awg_status set_error(awg_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

// Allocations left before an injected out-of-memory failure (-1: no injection), and the number
// of live device allocations.
static std::atomic<int64_t> g_fail_after{-1};
static std::atomic<int64_t> g_live_allocs{0};

cudaError_t dev_alloc_raw(void** p, size_t bytes) {
  int64_t left = g_fail_after.load();
  while (left >= 0) {
    if (left == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  return e;
}

void dev_free(void* p) {
  if (!p) return;
  cudaFree(p);
  g_live_allocs.fetch_sub(1);
}

awg_status cuda_error(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(AWG_ERR_OOM, std::string("device allocation failed in ") + where);
  }
  return set_error(AWG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

static float bf16_to_f32(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

static awg_status check_params(const awg_cf_params* p, bool from_table) {
  if (!p) return set_error(AWG_ERR_INVALID_ARG, "params is NULL");
  if (p->grid_n < 16 || p->grid_n > 65536 || (p->grid_n & 1))
    return set_error(AWG_ERR_INVALID_ARG, "grid_n must be even and in [16, 65536]");
  if (p->oversampling < 1 || p->oversampling > 250)
    return set_error(AWG_ERR_INVALID_ARG, "oversampling must be in [1, 250]");
  if (p->n_pa_bins < 1 || p->n_subbands < 1 || p->n_pa_bins * p->n_subbands > 1 << 20)
    return set_error(AWG_ERR_INVALID_ARG, "n_pa_bins and n_subbands must be >= 1");
  if (p->use_w && (p->n_wplanes < 2 || !(p->w_max_lambda > 0.0)))
    return set_error(AWG_ERR_INVALID_ARG, "use_w needs n_wplanes >= 2 and w_max_lambda > 0");
  if (p->cf_dtype != AWG_CF_FP32 && p->cf_dtype != AWG_CF_BF16)
    return set_error(AWG_ERR_INVALID_ARG, "cf_dtype must be AWG_CF_FP32 or AWG_CF_BF16");
  if (from_table) return AWG_OK;
  if (!(p->cell_rad > 0.0) || p->cell_rad * p->grid_n >= 2.0)
    return set_error(AWG_ERR_INVALID_ARG, "cell_rad must be > 0 with the field inside the sky");
  if (p->use_ps && p->ps_support < 1) return set_error(AWG_ERR_INVALID_ARG, "ps_support must be >= 1");
  if (p->max_support < 1) return set_error(AWG_ERR_INVALID_ARG, "max_support must be >= 1");
  if (p->max_support > kMaxSupport) return set_error(AWG_ERR_UNSUPPORTED, "max_support > 64 is not supported");
  if (p->use_ps && p->ps_support > p->max_support)
    return set_error(AWG_ERR_INVALID_ARG, "ps_support must not exceed max_support");
  if (p->use_a) {
    if (!p->pa_bin_centers_rad || !p->subband_freq_hz)
      return set_error(AWG_ERR_INVALID_ARG, "use_a needs pa_bin_centers_rad and subband_freq_hz");
    if (!(p->dish_diameter_m > 0.0) || !(std::fabs(p->ellipticity) < 0.5))
      return set_error(AWG_ERR_INVALID_ARG, "dish_diameter_m must be > 0 and |ellipticity| < 0.5");
  }
  if (p->use_pol) {
    if (!p->use_a) return set_error(AWG_ERR_INVALID_ARG, "use_pol needs use_a");
    if (!p->separable || p->cf_dtype != AWG_CF_FP32)
      return set_error(AWG_ERR_UNSUPPORTED, "full-polarisation CF sets need separable FP32 storage");
    if (!(std::fabs(p->squint_rad) < 0.1) || !(std::hypot(p->leakage_re, p->leakage_im) < 1.0) ||
        !(p->mueller_threshold >= 0.0))
      return set_error(AWG_ERR_INVALID_ARG, "need |squint_rad| < 0.1, |leakage| < 1 and mueller_threshold >= 0");
  }
  return AWG_OK;
}

void fill_slots(CfSetImpl* cf) {
  bool present[kMaxSupport + 1] = {false};
  for (int s : cf->supports) present[s] = true;
  SlotTable& st = cf->slots;
  st = SlotTable{};
  for (int s = 0; s <= kMaxSupport; ++s) st.slot_of_S[s] = -1;
  const int N = cf->p.grid_n;
  int base = 0;
  for (int s = 1; s <= kMaxSupport; ++s) {
    if (!present[s]) continue;
    const int i = st.n++;
    st.S[i] = s;
    st.tile[i] = cf->separable && has_exact(s) ? exact_cfg(s, cf->cand[s]).tile : kClasses[class_of_support(s)].tile;
    const int span = N - s + 1;    // possible first-tap positions per axis
    st.nt[i] = span > 0 ? (span + st.tile[i] - 1) / st.tile[i] : 0;
    st.base[i] = base;
    st.slot_of_S[s] = i;
    base += st.nt[i] * st.nt[i];
  }
  st.base[st.n] = base;
  cf->slots_version += 1;
}

static void free_cf(CfSetImpl* cf) {
  if (!cf) return;
  dev_free(cf->d_data);
  dev_free(cf->d_off);
  dev_free(cf->d_sup);
  dev_free(cf->d_inv_taper);
  dev_free(cf->d_sep);
  dev_free(cf->d_sep_off);
  dev_free(cf->d_mix);
  delete cf;
}

// Upload the host tables of one batch (FP64 interleaved) into the device array at their offsets.
static awg_status upload_tables(CfSetImpl* cf, const std::vector<int>& idx, const std::vector<std::vector<double>>& tabs,
                                cudaStream_t st) {
  const bool bf16 = cf->p.cf_dtype == AWG_CF_BF16;
  for (size_t j = 0; j < idx.size(); ++j) {
    const int ci = idx[j];
    const int64_t nv = (int64_t)tabs[j].size() / 2;
    if (bf16) {
      std::vector<uint16_t> h((size_t)nv * 2);
      for (int64_t i = 0; i < 2 * nv; ++i) h[i] = f32_to_bf16_rne((float)tabs[j][i]);
      AWG_CUDA_TRY(cudaMemcpyAsync((uint16_t*)cf->d_data + 2 * cf->offsets[ci], h.data(), 4 * nv,
                                   cudaMemcpyHostToDevice, st));
      AWG_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      std::vector<float> h((size_t)nv * 2);
      for (int64_t i = 0; i < 2 * nv; ++i) h[i] = (float)tabs[j][i];
      AWG_CUDA_TRY(cudaMemcpyAsync((float*)cf->d_data + 2 * cf->offsets[ci], h.data(), 8 * nv,
                                   cudaMemcpyHostToDevice, st));
      AWG_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }
  return AWG_OK;
}

static awg_status alloc_cf(CfSetImpl* cf, cudaStream_t st) {
  cf->n_signed = cf->p.use_w ? 2 * cf->p.n_wplanes - 1 : 1;
  cf->offsets.resize(cf->n_cf);
  int64_t off = 0;
  const int64_t per = (int64_t)(cf->p.oversampling + 1) * (cf->p.oversampling + 1);
  for (int i = 0; i < cf->n_cf; ++i) {
    cf->offsets[i] = off;
    off += per * cf->supports[i] * cf->supports[i];
  }
  cf->n_values = off;
  const size_t bytes = (size_t)off * (cf->p.cf_dtype == AWG_CF_BF16 ? 4 : 8);
  size_t free_b = 0, total_b = 0;
  AWG_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (bytes + (size_t)(256u << 20) > free_b)
    return set_error(AWG_ERR_OOM, "CF set of " + std::to_string(bytes >> 20) + " MiB does not fit in device memory");
  AWG_CUDA_TRY(dev_alloc(&cf->d_data, bytes));
  AWG_CUDA_TRY(dev_alloc(&cf->d_off, sizeof(int64_t) * cf->n_cf));
  AWG_CUDA_TRY(dev_alloc(&cf->d_sup, sizeof(int32_t) * cf->n_cf));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_off, cf->offsets.data(), sizeof(int64_t) * cf->n_cf, cudaMemcpyHostToDevice, st));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_sup, cf->supports.data(), sizeof(int32_t) * cf->n_cf, cudaMemcpyHostToDevice, st));
  std::vector<double> taper;
  taper_image(cf->p, taper);
  std::vector<float> inv(cf->p.grid_n);
  for (int i = 0; i < cf->p.grid_n; ++i) inv[i] = (float)(1.0 / taper[i]);
  AWG_CUDA_TRY(dev_alloc(&cf->d_inv_taper, sizeof(float) * cf->p.grid_n));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_inv_taper, inv.data(), sizeof(float) * cf->p.grid_n, cudaMemcpyHostToDevice, st));
  AWG_CUDA_TRY(cudaStreamSynchronize(st));
  fill_slots(cf);
  return AWG_OK;
}

// Upload the factors of every CF as the separable storage, with the support / offset bookkeeping
// the plan shares with the 2-D layout.  fx[ci], fy[ci] hold the CF's terms back to back (FP64
// pairs, [(OS+1) S] per term); the set's rank is the largest term count, and a CF with fewer
// terms gets zero terms (all of them point at one zero block at the start of the storage).
static awg_status upload_separable(CfSetImpl* cf, const std::vector<std::vector<double>>& fx,
                                   const std::vector<std::vector<double>>& fy, cudaStream_t st) {
  const int OS = cf->p.oversampling;
  int rank = 1;
  for (int i = 0; i < cf->n_cf; ++i)
    rank = std::max(rank, (int)(fx[i].size() / (2 * (size_t)(OS + 1) * cf->supports[i])));
  cf->separable = 1;
  cf->rank = rank;
  // fused kernels (one plan record per sample) for 2..4 terms on the exact supports; otherwise the
  // plan holds one record per sample and term
  cf->fused = rank >= 2 && rank <= 4 ? rank : 0;
  for (int i = 0; i < cf->n_cf && cf->fused; ++i)
    if (!has_exact(cf->supports[i])) cf->fused = 0;
  cf->sep_offsets.assign((size_t)cf->n_cf * rank, 0);
  int64_t off = 2 * (int64_t)(OS + 1) * kMaxSupport;   // the zero block (fx and fy of the largest support)
  for (int i = 0; i < cf->n_cf; ++i) {
    const int64_t q = (int64_t)(OS + 1) * cf->supports[i];
    const int r_i = (int)(fx[i].size() / (2 * q));
    for (int k = 0; k < r_i; ++k) {
      cf->sep_offsets[(size_t)i * rank + k] = off;
      off += 2 * q;
    }
  }
  cf->n_values = off;
  std::vector<float> h((size_t)2 * off, 0.f);
  for (int i = 0; i < cf->n_cf; ++i) {
    const int64_t q = (int64_t)(OS + 1) * cf->supports[i];
    const int r_i = (int)(fx[i].size() / (2 * q));
    for (int k = 0; k < r_i; ++k) {
      const int64_t o = 2 * cf->sep_offsets[(size_t)i * rank + k];
      for (int64_t t = 0; t < 2 * q; ++t) {
        h[o + t] = (float)fx[i][2 * q * k + t];
        h[o + 2 * q + t] = (float)fy[i][2 * q * k + t];
      }
    }
  }
  AWG_CUDA_TRY(dev_alloc(&cf->d_sep, sizeof(float) * h.size()));
  AWG_CUDA_TRY(dev_alloc(&cf->d_sep_off, sizeof(int64_t) * cf->sep_offsets.size()));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_sep, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_sep_off, cf->sep_offsets.data(), sizeof(int64_t) * cf->sep_offsets.size(),
                               cudaMemcpyHostToDevice, st));
  // the support / offset bookkeeping the plan and the kernels share with the 2-D layout
  AWG_CUDA_TRY(dev_alloc(&cf->d_sup, sizeof(int32_t) * cf->n_cf));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_sup, cf->supports.data(), sizeof(int32_t) * cf->n_cf, cudaMemcpyHostToDevice, st));
  std::vector<double> taper;
  taper_image(cf->p, taper);
  std::vector<float> inv(cf->p.grid_n);
  for (int i = 0; i < cf->p.grid_n; ++i) inv[i] = (float)(1.0 / taper[i]);
  AWG_CUDA_TRY(dev_alloc(&cf->d_inv_taper, sizeof(float) * cf->p.grid_n));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_inv_taper, inv.data(), sizeof(float) * cf->p.grid_n, cudaMemcpyHostToDevice, st));
  AWG_CUDA_TRY(cudaStreamSynchronize(st));
  fill_slots(cf);
  return AWG_OK;
}

// Separable storage: fit every non-negative plane as a sum of at most kMaxRank outer products
// fy fx (from its image-plane screen, without forming the 2-D table), mirror the fit for the
// negative planes, upload only the factors.  Returns AWG_ERR_UNSUPPORTED (nothing allocated on
// the device) when some CF needs more terms than that to come within kSepTol of its peak.
static awg_status upload_mix(CfSetImpl* cf, cudaStream_t st);

static awg_status build_separable(CfSetImpl* cf, cudaStream_t st) {
  const awg_cf_params& p = cf->p;
  cf->n_signed = p.use_w ? 2 * p.n_wplanes - 1 : 1;
  // The non-W part of every screen is real (the pol-shared A-term, or a base product of real
  // voltage patterns), so a negative-w plane is the conjugate point reflection of the positive one
  // and only n_w planes are fitted.
  const bool mirror = true;
  const int n_w = !p.use_w ? 1 : mirror ? p.n_wplanes : 2 * p.n_wplanes - 1;
  const int n_pos = p.n_pa_bins * p.n_subbands * n_w;
  const int OS = p.oversampling;
  std::vector<std::vector<double>> fx(cf->n_cf), fy(cf->n_cf);
  int failed = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int je = 0; je < n_pos * cf->n_mb; ++je) {
    if (failed) continue;
    const int e = je / n_pos, j = je - e * n_pos;
    const int k = j % n_w, pasb = j / n_w;
    const int pa = pasb / p.n_subbands, sb = pasb % p.n_subbands;
    const int ks = !p.use_w ? 0 : mirror ? p.n_wplanes - 1 + k : k;
    const int S = support_of_plane(p, ks);
    const int ci = e * cf->n_base + pasb * cf->n_signed + ks;
    // base block e of a full-polarisation set: the diagonal element of pol kBasePol[e], whose
    // screen is the voltage-pattern product A_a A_b itself
    const int ep = p.use_pol ? kBasePol[e] : -1, eq = ep;
    if (build_cf_factors(p, cf->pa_centers.data(), cf->sb_freqs.data(), pa, sb, ks, ep, eq, kSepTol, kMaxRank,
                         fx[ci], fy[ci]) == 0) {
#pragma omp atomic write
      failed = 1;
      continue;
    }
    if (mirror && p.use_w && k > 0) {
      // table(-w) = conj(table(+w)) point-reflected: each term's factors reversed and conjugated
      const int cn = e * cf->n_base + pasb * cf->n_signed + (p.n_wplanes - 1 - k);
      const size_t q = (size_t)(OS + 1) * S;
      const size_t terms = fx[ci].size() / (2 * q);
      fx[cn].resize(fx[ci].size());
      fy[cn].resize(fy[ci].size());
      for (size_t t = 0; t < terms; ++t)
        for (size_t i = 0; i < q; ++i) {
          const size_t d = 2 * (t * q + i), sidx = 2 * (t * q + q - 1 - i);
          fx[cn][d] = fx[ci][sidx];
          fx[cn][d + 1] = -fx[ci][sidx + 1];
          fy[cn][d] = fy[ci][sidx];
          fy[cn][d + 1] = -fy[ci][sidx + 1];
        }
    }
  }
  if (failed) return AWG_ERR_UNSUPPORTED;
  if (cf->n_mb > 1) {
    // base passes need the fused kernels (2..4 terms, exact supports); otherwise store every
    // element as s_pq times its base factors (fx scaled) for the single-pol element passes
    int rank = 1;
    bool exact = true;
    for (int i = 0; i < cf->n_cf; ++i) {
      rank = std::max(rank, (int)(fx[i].size() / (2 * (size_t)(OS + 1) * cf->supports[i])));
      exact = exact && has_exact(cf->supports[i]);
    }
    if (!(rank >= 2 && rank <= 4 && exact)) {
      std::vector<std::vector<double>> ex((size_t)cf->n_elem * cf->n_base), ey(ex.size());
      for (int e = 0; e < cf->n_elem; ++e) {
        const double sr = cf->elem_s[e][0], si = cf->elem_s[e][1];
        for (int c = 0; c < cf->n_base; ++c) {
          const size_t b = (size_t)cf->elem_mb[e] * cf->n_base + c, d = (size_t)e * cf->n_base + c;
          ex[d] = fx[b];
          ey[d] = fy[b];
          for (size_t t = 0; t + 1 < ex[d].size(); t += 2) {
            const double re = ex[d][t], im = ex[d][t + 1];
            ex[d][t] = sr * re - si * im;
            ex[d][t + 1] = sr * im + si * re;
          }
        }
      }
      fx.swap(ex);
      fy.swap(ey);
      cf->n_mb = cf->n_elem;
      cf->mb_elements = 1;
      cf->n_cf = cf->n_elem * cf->n_base;
      std::vector<int32_t> sup((size_t)cf->n_cf);
      for (int i = 0; i < cf->n_cf; ++i) sup[i] = cf->supports[i % cf->n_base];
      cf->supports.swap(sup);
    }
  }
  awg_status s = upload_separable(cf, fx, fy, st);
  if (s != AWG_OK || cf->n_mb == 1 || cf->mb_elements) return s;
  return upload_mix(cf, st);
}

// The pol-mixing matrices of the base blocks of a full-polarisation set: gridding
// mix_g[4 q + p] = conj(s_pq), degridding mix_d[4 p + q] = s_pq, for the kept elements (p, q) of
// the block.
static awg_status upload_mix(CfSetImpl* cf, cudaStream_t st) {
  std::vector<float2> mix((size_t)cf->n_mb * 32, make_float2(0.f, 0.f));
  for (int e = 0; e < cf->n_elem; ++e) {
    const int k = cf->elem_mb[e], pp = cf->elem_p[e], qq = cf->elem_q[e];
    const float sr = (float)cf->elem_s[e][0], si = (float)cf->elem_s[e][1];
    mix[(size_t)k * 32 + 4 * qq + pp] = make_float2(sr, -si);
    mix[(size_t)k * 32 + 16 + 4 * pp + qq] = make_float2(sr, si);
  }
  AWG_CUDA_TRY(dev_alloc(&cf->d_mix, sizeof(float2) * mix.size()));
  AWG_CUDA_TRY(cudaMemcpyAsync(cf->d_mix, mix.data(), sizeof(float2) * mix.size(), cudaMemcpyHostToDevice, st));
  AWG_CUDA_TRY(cudaStreamSynchronize(st));
  return AWG_OK;
}

// A CF set's host state from checked params: the A-term bin centres and frequencies, the Mueller
// elements with their base blocks and scalars, and the support of every stored CF (no device
// memory yet).  NULL when the host allocation fails.
static CfSetImpl* new_cf_set(const awg_cf_params* params) {
  CfSetImpl* cf = new (std::nothrow) CfSetImpl();
  if (!cf) return nullptr;
  cf->p = *params;
  if (params->use_a) {
    cf->pa_centers.assign(params->pa_bin_centers_rad, params->pa_bin_centers_rad + params->n_pa_bins);
    cf->sb_freqs.assign(params->subband_freq_hz, params->subband_freq_hz + params->n_subbands);
  }
  cf->p.pa_bin_centers_rad = nullptr;
  cf->p.subband_freq_hz = nullptr;
  cudaGetDevice(&cf->device);
  const int n_signed = params->use_w ? 2 * params->n_wplanes - 1 : 1;
  cf->n_signed = n_signed;
  cf->n_base = params->n_pa_bins * params->n_subbands * n_signed;
  cf->n_elem = params->use_pol ? mueller_elements(cf->p, cf->elem_p, cf->elem_q) : 1;
  if (params->use_pol) {
    // element (p, q), p = (a, b), q = (c, e): J_ac conj(J_be) = A_a A_b f(a, c) conj(f(b, e)) with
    // f(x, y) = 1 for x == y, else the leakage d: base block a + b, scalar f(a, c) conj(f(b, e))
    cf->n_mb = 3;
    const std::complex<double> d(params->leakage_re, params->leakage_im);
    for (int e = 0; e < cf->n_elem; ++e) {
      const int pp = cf->elem_p[e], qq = cf->elem_q[e];
      const int a = pp >> 1, b = pp & 1, c = qq >> 1, ee = qq & 1;
      const std::complex<double> s = (a == c ? 1.0 : d) * std::conj(b == ee ? std::complex<double>(1.0) : d);
      cf->elem_mb[e] = a + b;
      cf->elem_s[e][0] = s.real();
      cf->elem_s[e][1] = s.imag();
      cf->mb_pmask[a + b] |= 1 << pp;
    }
  }
  cf->n_cf = cf->n_mb * cf->n_base;
  cf->supports.resize(cf->n_cf);
  for (int e = 0; e < cf->n_mb; ++e)
    for (int pa = 0; pa < params->n_pa_bins; ++pa)
      for (int sb = 0; sb < params->n_subbands; ++sb)
        for (int ks = 0; ks < n_signed; ++ks)
          cf->supports[e * cf->n_base + (pa * params->n_subbands + sb) * n_signed + ks] = support_of_plane(cf->p, ks);
  return cf;
}

}  // namespace awg

using namespace awg;

extern "C" {

awg_status awg_debug_fail_allocations(int64_t after) {
  if (after < -1) return set_error(AWG_ERR_INVALID_ARG, "after must be >= -1");
  g_fail_after.store(after);
  return AWG_OK;
}

int64_t awg_debug_live_allocations(void) { return g_live_allocs.load(); }

const char* awg_last_error(void) { return g_last_error.c_str(); }

int64_t awg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

awg_status cf_set_create(const awg_cf_params* params, void* stream, awg_cf_set* out) {
  NvtxRange nvtx_range("awg cf_set_create (CF build)");
  if (!out) return set_error(AWG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  awg_status s = check_params(params, false);
  if (s != AWG_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  CfSetImpl* cf = new_cf_set(params);
  if (!cf) return set_error(AWG_ERR_OOM, "host allocation failed");
  const int n_signed = cf->n_signed;
  if (params->separable && params->cf_dtype == AWG_CF_FP32) {
    s = build_separable(cf, st);
    if (s == AWG_OK) {
      *out = (awg_cf_set)cf;
      return AWG_OK;
    }
    if (s != AWG_ERR_UNSUPPORTED || params->use_pol) {
      free_cf(cf);
      return s == AWG_ERR_UNSUPPORTED ? set_error(s, "a Mueller element CF needs more than 6 terms") : s;
    }
    cf->separable = 0;   // some CF is not an outer product: keep full tables
  }
  s = alloc_cf(cf, st);
  if (s != AWG_OK) { free_cf(cf); return s; }
  // Build the non-negative planes (the others are their conjugate point reflections) in batches
  // of bounded host memory, OpenMP over CFs within a batch.
  const int n_w = params->use_w ? params->n_wplanes : 1;
  const int n_pos = params->n_pa_bins * params->n_subbands * n_w;
  const int64_t per = (int64_t)(params->oversampling + 1) * (params->oversampling + 1);
  const int64_t budget = (int64_t)1 << 31;   // FP64 values per batch (16 GiB of host memory)
  int j0 = 0;
  while (j0 < n_pos) {
    std::vector<int> jobs;
    int64_t used = 0;
    for (int j = j0; j < n_pos; ++j) {
      const int k = j % n_w;
      const int ks = params->use_w ? params->n_wplanes - 1 + k : 0;
      const int S = support_of_plane(cf->p, ks);
      const int64_t need = 2 * per * S * S * (params->use_w && k > 0 ? 2 : 1);
      if (!jobs.empty() && used + need > budget) break;
      jobs.push_back(j);
      used += need;
    }
    std::vector<std::vector<double>> tabs(jobs.size());
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < (int)jobs.size(); ++q) {
      const int j = jobs[q];
      const int k = j % n_w, pasb = j / n_w;
      const int pa = pasb / params->n_subbands, sb = pasb % params->n_subbands;
      const int ks = params->use_w ? params->n_wplanes - 1 + k : 0;
      build_cf_table(cf->p, cf->pa_centers.data(), cf->sb_freqs.data(), pa, sb, ks, tabs[q]);
    }
    std::vector<int> idx;
    std::vector<std::vector<double>> all;
    for (size_t q = 0; q < jobs.size(); ++q) {
      const int j = jobs[q];
      const int k = j % n_w, pasb = j / n_w;
      const int ks = params->use_w ? params->n_wplanes - 1 + k : 0;
      const bool has_neg = params->use_w && k > 0;
      std::vector<double> neg;
      if (has_neg) {
        // table(-w)[o][t] = conj(table(+w)[OS - o][S - 1 - t]): the flat array reversed, conjugated.
        const std::vector<double>& t = tabs[q];
        const size_t nv = t.size() / 2;
        neg.resize(t.size());
        for (size_t i = 0; i < nv; ++i) {
          neg[2 * i] = t[2 * (nv - 1 - i)];
          neg[2 * i + 1] = -t[2 * (nv - 1 - i) + 1];
        }
      }
      idx.push_back(pasb * n_signed + ks);
      all.push_back(std::move(tabs[q]));
      if (has_neg) {
        idx.push_back(pasb * n_signed + (params->n_wplanes - 1 - k));
        all.push_back(std::move(neg));
      }
    }
    s = upload_tables(cf, idx, all, st);
    if (s != AWG_OK) { free_cf(cf); return s; }
    j0 += (int)jobs.size();
  }
  *out = (awg_cf_set)cf;
  return AWG_OK;
}

awg_status cf_set_create_from_table(const awg_cf_params* params, const int32_t* supports, const float* table,
                                    void* stream, awg_cf_set* out) {
  if (!out) return set_error(AWG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  awg_status s = check_params(params, true);
  if (s != AWG_OK) return s;
  if (params->use_pol) return set_error(AWG_ERR_UNSUPPORTED, "caller tables cannot form a Mueller set");
  if (!supports || !table) return set_error(AWG_ERR_INVALID_ARG, "supports and table must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  CfSetImpl* cf = new (std::nothrow) CfSetImpl();
  if (!cf) return set_error(AWG_ERR_OOM, "host allocation failed");
  cf->p = *params;
  cf->p.pa_bin_centers_rad = nullptr;
  cf->p.subband_freq_hz = nullptr;
  cf->p.use_ps = 0;
  cf->p.use_a = 0;
  cudaGetDevice(&cf->device);
  const int n_signed = params->use_w ? 2 * params->n_wplanes - 1 : 1;
  cf->n_cf = params->n_pa_bins * params->n_subbands * n_signed;
  cf->n_base = cf->n_cf;
  cf->supports.assign(supports, supports + cf->n_cf);
  for (int v : cf->supports) {
    if (v < 1) { delete cf; return set_error(AWG_ERR_INVALID_ARG, "supports must be >= 1"); }
    if (v > kMaxSupport) { delete cf; return set_error(AWG_ERR_UNSUPPORTED, "support > 64 is not supported"); }
    if (v > params->grid_n) { delete cf; return set_error(AWG_ERR_INVALID_ARG, "support exceeds grid_n"); }
  }
  if (params->separable && params->cf_dtype == AWG_CF_FP32) {
    // keep only factors when every caller table is an outer product to FP32 accuracy
    cf->n_signed = params->use_w ? 2 * params->n_wplanes - 1 : 1;
    int64_t off = 0;
    std::vector<int64_t> offs(cf->n_cf);
    for (int ci = 0; ci < cf->n_cf; ++ci) {
      offs[ci] = off;
      off += (int64_t)(params->oversampling + 1) * (params->oversampling + 1) * cf->supports[ci] * cf->supports[ci];
    }
    std::vector<std::vector<double>> fx(cf->n_cf), fy(cf->n_cf);
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int ci = 0; ci < cf->n_cf; ++ci) {
      if (failed) continue;
      const int S = cf->supports[ci];
      const int64_t nv = (int64_t)(params->oversampling + 1) * (params->oversampling + 1) * S * S;
      std::vector<double> tab(table + 2 * offs[ci], table + 2 * (offs[ci] + nv));
      if (factor_low_rank(tab, S, params->oversampling, kSepTol, kMaxRank, fx[ci], fy[ci]) == 0) {
#pragma omp atomic write
        failed = 1;
      }
    }
    if (!failed) {
      s = upload_separable(cf, fx, fy, st);
      if (s != AWG_OK) { free_cf(cf); return s; }
      *out = (awg_cf_set)cf;
      return AWG_OK;
    }
  }
  s = alloc_cf(cf, st);
  if (s != AWG_OK) { free_cf(cf); return s; }
  std::vector<int> idx;
  std::vector<std::vector<double>> all;
  for (int ci = 0; ci < cf->n_cf; ++ci) {
    const int64_t nv = (int64_t)(params->oversampling + 1) * (params->oversampling + 1) * cf->supports[ci] * cf->supports[ci];
    const float* src = table + 2 * cf->offsets[ci];
    idx.push_back(ci);
    all.emplace_back(src, src + 2 * nv);
    if (all.size() >= 64 || ci == cf->n_cf - 1) {
      s = upload_tables(cf, idx, all, st);
      if (s != AWG_OK) { free_cf(cf); return s; }
      idx.clear();
      all.clear();
    }
  }
  *out = (awg_cf_set)cf;
  return AWG_OK;
}

awg_status cf_set_destroy(awg_cf_set h) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "cf set is NULL");
  free_cf((CfSetImpl*)h);
  return AWG_OK;
}

awg_status cf_set_autotune(awg_cf_set h, const double* uvw_m, int64_t n_rows, const double* freq_hz, int32_t n_chan,
                           const int32_t* pa_bin, const int32_t* chan_subband, int32_t n_pol, void* stream,
                           int32_t* choice_out, float* ms_out) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "cf set is NULL");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (n_pol != 1 && n_pol != 2 && n_pol != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  if (n_rows < 0 || n_chan < 1) return set_error(AWG_ERR_INVALID_ARG, "n_rows must be >= 0 and n_chan >= 1");
  if (n_rows > 0 && (!uvw_m || !freq_hz)) return set_error(AWG_ERR_INVALID_ARG, "uvw_m and freq_hz must not be NULL");
  if (cf->p.n_pa_bins > 1 && !pa_bin) return set_error(AWG_ERR_INVALID_ARG, "pa_bin is required with n_pa_bins > 1");
  if (cf->p.n_subbands > 1 && !chan_subband)
    return set_error(AWG_ERR_INVALID_ARG, "chan_subband is required with n_subbands > 1");
  if (cudaSetDevice(cf->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  int32_t choice[kMaxSupport + 1];
  awg_status s = autotune_supports(cf, uvw_m, n_rows, freq_hz, n_chan, pa_bin, chan_subband, n_pol,
                                   (cudaStream_t)stream, choice, ms_out);
  if (choice_out) std::memcpy(choice_out, choice, sizeof(choice));
  return s;
}

awg_status cf_set_choose(awg_cf_set h, int32_t support, int32_t config) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "cf set is NULL");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (support < 1 || support > kMaxSupport || !has_exact(support))
    return set_error(AWG_ERR_INVALID_ARG, "support " + std::to_string(support) + " has no kernel configurations");
  if (config < 0 || config >= kNumCand) return set_error(AWG_ERR_INVALID_ARG, "config must be 0, 1, 2 or 3");
  if (cf->fused && (config > 1 || (config == 1 && cf->n_mb > 1)))
    return set_error(AWG_ERR_UNSUPPORTED, cf->n_mb > 1 ? "pol-mixing kernels have one configuration"
                                                       : "fused kernels have configurations 0 and 1");
  cf->cand[support] = (int8_t)config;
  fill_slots(cf);
  return AWG_OK;
}

awg_status cf_set_mueller(awg_cf_set h, int32_t* n_elem, int32_t* elem_p, int32_t* elem_q) {
  if (!h || !n_elem) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)h;
  *n_elem = cf->p.use_pol ? cf->n_elem : 0;
  for (int e = 0; e < *n_elem; ++e) {
    if (elem_p) elem_p[e] = cf->elem_p[e];
    if (elem_q) elem_q[e] = cf->elem_q[e];
  }
  return AWG_OK;
}

awg_status cf_set_info(awg_cf_set h, int32_t* n_cf, int64_t* n_values, int32_t* separable) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "cf set is NULL");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (n_cf) *n_cf = cf->p.use_pol ? cf->n_elem * cf->n_base : cf->n_cf;   // Mueller sets: element-major
  if (n_values) *n_values = cf->n_values;
  if (separable) *separable = cf->separable ? cf->rank : 0;
  return AWG_OK;
}

awg_status cf_set_fused_terms(awg_cf_set h, int32_t* terms) {
  if (!h || !terms) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)h;
  *terms = cf->fused;
  return AWG_OK;
}

awg_status cf_set_get_params(awg_cf_set h, awg_cf_params* out, double* pa_bin_centers_rad, double* subband_freq_hz) {
  if (!h || !out) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  const CfSetImpl* cf = (const CfSetImpl*)h;
  *out = cf->p;
  out->pa_bin_centers_rad = nullptr;
  out->subband_freq_hz = nullptr;
  if (pa_bin_centers_rad && !cf->pa_centers.empty())
    std::memcpy(pa_bin_centers_rad, cf->pa_centers.data(), sizeof(double) * cf->pa_centers.size());
  if (subband_freq_hz && !cf->sb_freqs.empty())
    std::memcpy(subband_freq_hz, cf->sb_freqs.data(), sizeof(double) * cf->sb_freqs.size());
  return AWG_OK;
}

// CF cache file (same-endian hosts): magic, format version, sizeof(awg_cf_params), the params
// (pointers zeroed), the A-term bin centres and frequencies, the storage mode (separable, blocks,
// element blocks, stored CFs), the support of every stored CF, the autotuned kernel choice per
// support, then either every stored CF's terms (count, then fx and fy of each term as FP32
// [OS+1][S] complex) or the raw table data, and an end marker.
static const char kCacheMagic[8] = {'A', 'W', 'G', 'C', 'F', 'S', 'E', 'T'};
static const char kCacheEnd[8] = {'A', 'W', 'G', 'C', 'F', 'E', 'N', 'D'};
static const int32_t kCacheVersion = 1;

awg_status cf_set_save(awg_cf_set h, const char* path) {
  if (!h || !path) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (cudaSetDevice(cf->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  // the device data first, so that a CUDA error leaves no partial file behind
  std::vector<float> sep;
  std::vector<unsigned char> raw;
  if (cf->separable) {
    sep.resize((size_t)2 * cf->n_values);
    AWG_CUDA_TRY(cudaMemcpy(sep.data(), cf->d_sep, sizeof(float) * sep.size(), cudaMemcpyDeviceToHost));
  } else {
    raw.resize((size_t)cf->n_values * (cf->p.cf_dtype == AWG_CF_BF16 ? 4 : 8));
    AWG_CUDA_TRY(cudaMemcpy(raw.data(), cf->d_data, raw.size(), cudaMemcpyDeviceToHost));
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(AWG_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
  bool ok = true;
  auto put = [&](const void* p, size_t n) { ok = ok && (n == 0 || std::fwrite(p, 1, n, f) == n); };
  awg_cf_params pp = cf->p;
  pp.pa_bin_centers_rad = nullptr;
  pp.subband_freq_hz = nullptr;
  const int32_t psize = (int32_t)sizeof(awg_cf_params);
  put(kCacheMagic, 8);
  put(&kCacheVersion, 4);
  put(&psize, 4);
  put(&pp, sizeof(pp));
  const int64_t n_pa = (int64_t)cf->pa_centers.size(), n_sb = (int64_t)cf->sb_freqs.size();
  put(&n_pa, 8);
  put(cf->pa_centers.data(), sizeof(double) * n_pa);
  put(&n_sb, 8);
  put(cf->sb_freqs.data(), sizeof(double) * n_sb);
  const int32_t mode[4] = {cf->separable, cf->n_mb, cf->mb_elements, cf->n_cf};
  put(mode, sizeof(mode));
  put(cf->supports.data(), sizeof(int32_t) * cf->n_cf);
  put(cf->cand, sizeof(cf->cand));
  if (cf->separable) {
    const int OS = cf->p.oversampling;
    for (int i = 0; i < cf->n_cf && ok; ++i) {
      const int64_t q = (int64_t)(OS + 1) * cf->supports[i];
      int32_t terms = 0;
      for (int k = 0; k < cf->rank; ++k) terms += cf->sep_offsets[(size_t)i * cf->rank + k] != 0;
      put(&terms, 4);
      for (int k = 0; k < cf->rank; ++k) {
        const int64_t o = cf->sep_offsets[(size_t)i * cf->rank + k];
        if (o != 0) put(sep.data() + 2 * o, sizeof(float) * 4 * q);   // fx then fy
      }
    }
  } else {
    put(raw.data(), raw.size());
  }
  put(kCacheEnd, 8);
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return set_error(AWG_ERR_INVALID_ARG, std::string("writing ") + path + " failed");
  return AWG_OK;
}

awg_status cf_set_load(const char* path, void* stream, awg_cf_set* out) {
  NvtxRange nvtx_range("awg cf_set_load");
  if (!path || !out) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(AWG_ERR_INVALID_ARG, std::string("cannot open ") + path);
  bool ok = true;
  auto get = [&](void* p, size_t n) { ok = ok && (n == 0 || std::fread(p, 1, n, f) == n); return ok; };
  auto fail = [&](const std::string& why) {
    std::fclose(f);
    return set_error(AWG_ERR_INVALID_ARG, std::string(path) + ": " + why);
  };
  char magic[8];
  int32_t version = 0, psize = 0;
  if (!get(magic, 8) || std::memcmp(magic, kCacheMagic, 8) != 0) return fail("not a CF cache file");
  if (!get(&version, 4) || version != kCacheVersion) return fail("unsupported CF cache version");
  if (!get(&psize, 4) || psize != (int32_t)sizeof(awg_cf_params)) return fail("CF parameter layout differs");
  awg_cf_params p;
  int64_t n_pa = 0, n_sb = 0;
  if (!get(&p, sizeof(p)) || !get(&n_pa, 8) || n_pa < 0 || n_pa > (1 << 20)) return fail("truncated or corrupt header");
  std::vector<double> pa((size_t)n_pa), sb;
  if (!get(pa.data(), sizeof(double) * n_pa) || !get(&n_sb, 8) || n_sb < 0 || n_sb > (1 << 20))
    return fail("truncated or corrupt header");
  sb.resize((size_t)n_sb);
  if (!get(sb.data(), sizeof(double) * n_sb)) return fail("truncated header");
  p.pa_bin_centers_rad = p.use_a ? pa.data() : nullptr;
  p.subband_freq_hz = p.use_a ? sb.data() : nullptr;
  if (p.use_a && (n_pa != p.n_pa_bins || n_sb != p.n_subbands)) return fail("A-term bins do not match the params");
  const bool from_table = !p.use_ps && !p.use_a;   // a caller-table set keeps its own supports
  if (check_params(&p, from_table) != AWG_OK) {
    const std::string why = g_last_error;
    return fail("invalid params: " + why);
  }
  int32_t mode[4];
  if (!get(mode, sizeof(mode))) return fail("truncated header");
  CfSetImpl* cf = new_cf_set(&p);
  if (!cf) {
    std::fclose(f);
    return set_error(AWG_ERR_OOM, "host allocation failed");
  }
  auto fail_cf = [&](const std::string& why) {
    free_cf(cf);
    return fail(why);
  };
  // the stored blocks: as built, or one block per Mueller element
  const bool elements = mode[2] != 0;
  if (elements) {
    if (!p.use_pol || mode[1] != cf->n_elem) return fail_cf("inconsistent storage mode");
    cf->n_mb = cf->n_elem;
    cf->mb_elements = 1;
    cf->n_cf = cf->n_elem * cf->n_base;
  } else if (mode[1] != cf->n_mb) {
    return fail_cf("inconsistent storage mode");
  }
  if (mode[3] != cf->n_cf || (mode[0] && !(p.separable && p.cf_dtype == AWG_CF_FP32)) || (p.use_pol && !mode[0]))
    return fail_cf("inconsistent storage mode");
  cf->supports.resize(cf->n_cf);
  if (!get(cf->supports.data(), sizeof(int32_t) * cf->n_cf) || !get(cf->cand, sizeof(cf->cand)))
    return fail_cf("truncated header");
  for (int i = 0; i < cf->n_cf; ++i)
    if (cf->supports[i] < 1 || cf->supports[i] > kMaxSupport) return fail_cf("corrupt supports");
  for (int S = 0; S <= kMaxSupport; ++S)
    if (cf->cand[S] < 0 || cf->cand[S] >= kNumCand || (cf->cand[S] && !has_exact(S))) return fail_cf("corrupt kernel choices");
  cudaStream_t st = (cudaStream_t)stream;
  awg_status s = AWG_OK;
  if (mode[0]) {
    const int OS = p.oversampling;
    std::vector<std::vector<double>> fx(cf->n_cf), fy(cf->n_cf);
    std::vector<float> buf;
    for (int i = 0; i < cf->n_cf; ++i) {
      const size_t q = (size_t)(OS + 1) * cf->supports[i];
      int32_t terms = 0;
      if (!get(&terms, 4) || terms < 1 || terms > kMaxRank) return fail_cf("corrupt factors");
      fx[i].resize(2 * q * terms);
      fy[i].resize(2 * q * terms);
      buf.resize(4 * q);
      for (int k = 0; k < terms; ++k) {
        if (!get(buf.data(), sizeof(float) * 4 * q)) return fail_cf("truncated factors");
        for (size_t t = 0; t < 2 * q; ++t) {
          fx[i][2 * q * k + t] = buf[t];
          fy[i][2 * q * k + t] = buf[2 * q + t];
        }
      }
    }
    char end[8];
    if (!get(end, 8) || std::memcmp(end, kCacheEnd, 8) != 0) return fail_cf("missing end marker");
    std::fclose(f);
    s = upload_separable(cf, fx, fy, st);
    if (s == AWG_OK && cf->n_mb > 1 && !cf->mb_elements) s = upload_mix(cf, st);
  } else {
    s = alloc_cf(cf, st);
    if (s != AWG_OK) {
      std::fclose(f);
      free_cf(cf);
      return s;
    }
    std::vector<unsigned char> raw((size_t)cf->n_values * (p.cf_dtype == AWG_CF_BF16 ? 4 : 8));
    char end[8];
    if (!get(raw.data(), raw.size()) || !get(end, 8) || std::memcmp(end, kCacheEnd, 8) != 0)
      return fail_cf("truncated tables");
    std::fclose(f);
    if (cudaMemcpy(cf->d_data, raw.data(), raw.size(), cudaMemcpyHostToDevice) != cudaSuccess) s = AWG_ERR_CUDA;
    if (s != AWG_OK) set_error(s, "uploading the tables failed");
  }
  if (s != AWG_OK) {   // the uploads above fill the slot table from the loaded kernel choices
    free_cf(cf);
    return s;
  }
  *out = (awg_cf_set)cf;
  return AWG_OK;
}

awg_status cf_set_get_supports(awg_cf_set h, int32_t* out) {
  if (!h || !out) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (cf->n_mb > 1 && !cf->mb_elements) {   // every element shares the supports of the base index
    for (int e = 0; e < cf->n_elem; ++e)
      std::memcpy(out + (size_t)e * cf->n_base, cf->supports.data(), sizeof(int32_t) * cf->n_base);
    return AWG_OK;
  }
  std::memcpy(out, cf->supports.data(), sizeof(int32_t) * cf->n_cf);
  return AWG_OK;
}

awg_status cf_set_copy_table(awg_cf_set h, int32_t ci, float* out) {
  if (!h || !out) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)h;
  // a Mueller element's CF is s_pq times its stored base CF
  float scale_r = 1.f, scale_i = 0.f;
  if (cf->n_mb > 1 && !cf->mb_elements) {
    if (ci < 0 || ci >= cf->n_elem * cf->n_base) return set_error(AWG_ERR_INVALID_ARG, "cf index out of range");
    const int e = ci / cf->n_base;
    scale_r = (float)cf->elem_s[e][0];
    scale_i = (float)cf->elem_s[e][1];
    ci = cf->elem_mb[e] * cf->n_base + ci % cf->n_base;
  }
  if (ci < 0 || ci >= cf->n_cf) return set_error(AWG_ERR_INVALID_ARG, "cf index out of range");
  const int64_t nv = (int64_t)(cf->p.oversampling + 1) * (cf->p.oversampling + 1) * cf->supports[ci] * cf->supports[ci];
  if (cf->separable) {
    // the sum of the CF's terms, each product in FP32 as the kernels form it
    const int OS = cf->p.oversampling, S = cf->supports[ci];
    const int64_t q = (int64_t)(OS + 1) * S;
    std::fill(out, out + 2 * nv, 0.f);
    std::vector<float> f((size_t)4 * q);
    for (int k = 0; k < cf->rank; ++k) {
      AWG_CUDA_TRY(cudaMemcpy(f.data(), (float*)cf->d_sep + 2 * cf->sep_offsets[(size_t)ci * cf->rank + k], 16 * q,
                              cudaMemcpyDeviceToHost));
      const float* fx = f.data();
      const float* fy = f.data() + 2 * q;
      for (int oy = 0; oy <= OS; ++oy)
        for (int ox = 0; ox <= OS; ++ox)
          for (int ty = 0; ty < S; ++ty)
            for (int tx = 0; tx < S; ++tx) {
              const float gr = fy[2 * (oy * S + ty)], gi = fy[2 * (oy * S + ty) + 1];
              const float fr = fx[2 * (ox * S + tx)], fi = fx[2 * (ox * S + tx) + 1];
              const size_t o = ((((size_t)oy * (OS + 1) + ox) * S + ty) * S + tx) * 2;
              out[o] += gr * fr - gi * fi;
              out[o + 1] += gr * fi + gi * fr;
            }
    }
    if (scale_r != 1.f || scale_i != 0.f)
      for (int64_t i = 0; i < nv; ++i) {
        const float re = out[2 * i], im = out[2 * i + 1];
        out[2 * i] = scale_r * re - scale_i * im;
        out[2 * i + 1] = scale_r * im + scale_i * re;
      }
    return AWG_OK;
  }
  if (cf->p.cf_dtype == AWG_CF_BF16) {
    std::vector<uint16_t> h16((size_t)2 * nv);
    AWG_CUDA_TRY(cudaMemcpy(h16.data(), (uint16_t*)cf->d_data + 2 * cf->offsets[ci], 4 * nv, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < 2 * nv; ++i) out[i] = bf16_to_f32(h16[i]);
  } else {
    AWG_CUDA_TRY(cudaMemcpy(out, (float*)cf->d_data + 2 * cf->offsets[ci], 8 * nv, cudaMemcpyDeviceToHost));
  }
  return AWG_OK;
}

awg_status cf_set_copy_factors(awg_cf_set h, int32_t ci, int32_t term, float* fx_out, float* fy_out,
                               float* scale_out) {
  if (!h || !fx_out || !fy_out) return set_error(AWG_ERR_INVALID_ARG, "NULL argument");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (!cf->separable) return set_error(AWG_ERR_INVALID_ARG, "the CF set holds full tables, not factors");
  if (term < 0 || term >= cf->rank) return set_error(AWG_ERR_INVALID_ARG, "term out of range");
  float scale_r = 1.f, scale_i = 0.f;
  if (cf->n_mb > 1 && !cf->mb_elements) {   // a Mueller element is s_pq times its stored base CF
    if (ci < 0 || ci >= cf->n_elem * cf->n_base) return set_error(AWG_ERR_INVALID_ARG, "cf index out of range");
    const int e = ci / cf->n_base;
    scale_r = (float)cf->elem_s[e][0];
    scale_i = (float)cf->elem_s[e][1];
    ci = cf->elem_mb[e] * cf->n_base + ci % cf->n_base;
  }
  if (ci < 0 || ci >= cf->n_cf) return set_error(AWG_ERR_INVALID_ARG, "cf index out of range");
  const int64_t q = (int64_t)(cf->p.oversampling + 1) * cf->supports[ci];
  const float* src = (const float*)cf->d_sep + 2 * cf->sep_offsets[(size_t)ci * cf->rank + term];
  AWG_CUDA_TRY(cudaMemcpy(fx_out, src, 8 * q, cudaMemcpyDeviceToHost));
  AWG_CUDA_TRY(cudaMemcpy(fy_out, src + 2 * q, 8 * q, cudaMemcpyDeviceToHost));
  if (scale_out) {
    scale_out[0] = scale_r;
    scale_out[1] = scale_i;
  }
  return AWG_OK;
}

static awg_status plan_free(PlanImpl* pl) {
  if (!pl) return AWG_OK;
  plan_free_side_streams(pl);
  dev_free(pl->d_rec);
  dev_free(pl->d_rec_tmp);
  dev_free(pl->d_part);
  dev_free(pl->d_key);
  dev_free(pl->d_drop);
  dev_free(pl->d_bcount);
  dev_free(pl->d_boff);
  dev_free(pl->d_icount);
  dev_free(pl->d_ioff);
  dev_free(pl->d_scan_tmp);
  dev_free(pl->d_items);
  dev_free(pl->d_class_range);
  dev_free(pl->d_slot_range);
  dev_free(pl->d_queue);
  dev_free(pl->d_counters);
  dev_free(pl->d_uvw);
  dev_free(pl->d_freq);
  dev_free(pl->d_row_dlm);
  dev_free(pl->d_phasor);
  delete pl;
  return AWG_OK;
}

awg_status plan_create(awg_cf_set h, const double* uvw_m, int64_t n_rows, const double* freq_hz, int32_t n_chan,
                       const int32_t* pa_bin, const int32_t* chan_subband, const double* phase_shift, void* stream,
                       awg_plan* out) {
  NvtxRange nvtx_range("awg plan_create");
  if (!out) return set_error(AWG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "cf set is NULL");
  CfSetImpl* cf = (CfSetImpl*)h;
  if (n_rows > 0 && (!uvw_m || !freq_hz)) return set_error(AWG_ERR_INVALID_ARG, "uvw_m and freq_hz must not be NULL");
  if (n_rows < 0 || n_chan < 1) return set_error(AWG_ERR_INVALID_ARG, "n_rows must be >= 0 and n_chan >= 1");
  if ((int64_t)n_rows * n_chan > ((int64_t)1 << 31) - 1)
    return set_error(AWG_ERR_UNSUPPORTED, "more than 2^31 - 1 samples per plan");
  if (cf->p.n_pa_bins > 1 && !pa_bin) return set_error(AWG_ERR_INVALID_ARG, "pa_bin is required with n_pa_bins > 1");
  if (cf->p.n_subbands > 1 && !chan_subband)
    return set_error(AWG_ERR_INVALID_ARG, "chan_subband is required with n_subbands > 1");
  PlanImpl* pl = new (std::nothrow) PlanImpl();
  if (!pl) return set_error(AWG_ERR_OOM, "host allocation failed");
  pl->cf = cf;
  pl->R = n_rows;
  pl->C = n_chan;
  pl->n = n_rows * n_chan;
  pl->rank = cf->separable && !cf->fused ? cf->rank : 1;
  pl->slots_version = cf->slots_version;
  pl->n_rec = pl->n * pl->rank;
  if (pl->n_rec > ((int64_t)1 << 31) - 1) {
    delete pl;
    return set_error(AWG_ERR_UNSUPPORTED, "more than 2^31 - 1 samples x CF terms per plan");
  }
  cudaGetDevice(&pl->device);
  if (phase_shift) {
    const double dl = phase_shift[0], dm = phase_shift[1];
    if (!(dl * dl + dm * dm < 1.0)) { delete pl; return set_error(AWG_ERR_INVALID_ARG, "phase shift outside the sky"); }
    pl->has_phase = 1;
    pl->global_phase = 1;
    pl->dl = dl;
    pl->dm = dm;
    pl->dn = std::sqrt(1.0 - dl * dl - dm * dm) - 1.0;
  }
  pl->n_buckets = cf->slots.base[cf->slots.n];
  pl->max_items = (int64_t)pl->n_buckets + pl->n_rec / kItemChunk + 1;
  const size_t n = (size_t)std::max<int64_t>(pl->n, 1);
  const size_t nr = (size_t)std::max<int64_t>(pl->n_rec, 1);
  const size_t nb = (size_t)pl->n_buckets + 1;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = dev_alloc(p, bytes); };
  A((void**)&pl->d_rec, nr * sizeof(SampleRec));
  A((void**)&pl->d_rec_tmp, nr * sizeof(SampleRec));
  A((void**)&pl->d_key, nr * sizeof(int32_t));
  A((void**)&pl->d_drop, n * sizeof(int32_t));
  if (pl->rank > 1) A((void**)&pl->d_part, nr * 4 * sizeof(float2));
  A((void**)&pl->d_bcount, nb * sizeof(int32_t));
  A((void**)&pl->d_boff, nb * sizeof(int32_t));
  A((void**)&pl->d_icount, nb * sizeof(int32_t));
  A((void**)&pl->d_ioff, nb * sizeof(int32_t));
  A((void**)&pl->d_scan_tmp, ((nb + 1023) / 1024 + 1024) * sizeof(int32_t));
  A((void**)&pl->d_items, (size_t)pl->max_items * sizeof(WorkItem));
  A((void**)&pl->d_class_range, (kNumClasses + 1) * sizeof(int32_t));
  A((void**)&pl->d_slot_range, (kMaxSupport + 1) * sizeof(int32_t));
  A((void**)&pl->d_queue, kMaxSupport * sizeof(int32_t));
  A((void**)&pl->d_counters, 4 * sizeof(unsigned long long));
  if (pl->has_phase) {
    A((void**)&pl->d_uvw, (size_t)std::max<int64_t>(pl->R, 1) * 3 * sizeof(double));
    A((void**)&pl->d_freq, (size_t)pl->C * sizeof(double));
    A((void**)&pl->d_phasor, n * sizeof(float2));
  }
  if (e != cudaSuccess) {
    plan_free(pl);
    return cuda_error(e, "plan_create allocation");
  }
  awg_status s = plan_make_side_streams(pl);
  if (s != AWG_OK) {
    plan_free(pl);
    return s;
  }
  s = plan_build(pl, uvw_m, freq_hz, pa_bin, chan_subband, (cudaStream_t)stream);
  if (s != AWG_OK) {
    plan_free(pl);
    return s;
  }
  *out = (awg_plan)pl;
  return AWG_OK;
}

awg_status plan_set_row_phase(awg_plan h, const double* row_dlm, const double* uvw_m, const double* freq_hz,
                              void* stream) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "plan is NULL");
  PlanImpl* pl = (PlanImpl*)h;
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  if (!row_dlm) {   // back to the plan-wide shift (or none)
    if (pl->d_row_dlm) {
      AWG_CUDA_TRY(cudaStreamSynchronize(st));
      dev_free(pl->d_row_dlm);
      pl->d_row_dlm = nullptr;
    }
    pl->has_phase = pl->global_phase;
    return pl->has_phase ? compute_phasors(pl, st) : AWG_OK;
  }
  if (pl->R > 0 && (!uvw_m || !freq_hz)) return set_error(AWG_ERR_INVALID_ARG, "uvw_m and freq_hz must not be NULL");
  const size_t R = (size_t)std::max<int64_t>(pl->R, 1);
  if (!pl->d_row_dlm) AWG_CUDA_TRY(dev_alloc(&pl->d_row_dlm, R * 2 * sizeof(double)));
  if (!pl->d_uvw) AWG_CUDA_TRY(dev_alloc(&pl->d_uvw, R * 3 * sizeof(double)));
  if (!pl->d_freq) AWG_CUDA_TRY(dev_alloc(&pl->d_freq, (size_t)pl->C * sizeof(double)));
  if (!pl->d_phasor) AWG_CUDA_TRY(dev_alloc(&pl->d_phasor, (size_t)std::max<int64_t>(pl->n, 1) * sizeof(float2)));
  if (pl->R > 0) {
    AWG_CUDA_TRY(cudaMemcpyAsync(pl->d_row_dlm, row_dlm, R * 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    AWG_CUDA_TRY(cudaMemcpyAsync(pl->d_uvw, uvw_m, R * 3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    AWG_CUDA_TRY(cudaMemcpyAsync(pl->d_freq, freq_hz, (size_t)pl->C * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  pl->has_phase = 1;
  return compute_phasors(pl, st);
}

awg_status plan_update(awg_plan h, const double* uvw_m, const double* freq_hz, const int32_t* pa_bin,
                       const int32_t* chan_subband, void* stream) {
  NvtxRange nvtx_range("awg plan_update");
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "plan is NULL");
  PlanImpl* pl = (PlanImpl*)h;
  if (pl->n > 0 && (!uvw_m || !freq_hz)) return set_error(AWG_ERR_INVALID_ARG, "uvw_m and freq_hz must not be NULL");
  if (pl->cf->p.n_pa_bins > 1 && !pa_bin) return set_error(AWG_ERR_INVALID_ARG, "pa_bin is required");
  if (pl->cf->p.n_subbands > 1 && !chan_subband) return set_error(AWG_ERR_INVALID_ARG, "chan_subband is required");
  if (pl->slots_version != pl->cf->slots_version)
    return set_error(AWG_ERR_INVALID_ARG, "the CF set was retuned after this plan was made; create a new plan");
  return plan_build(pl, uvw_m, freq_hz, pa_bin, chan_subband, (cudaStream_t)stream);
}

awg_status plan_destroy(awg_plan h) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "plan is NULL");
  return plan_free((PlanImpl*)h);
}

awg_status plan_stats(awg_plan h, int64_t* n_kept, int64_t* n_dropped, int64_t* sum_taps) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "plan is NULL");
  PlanImpl* pl = (PlanImpl*)h;
  unsigned long long c[4];
  AWG_CUDA_TRY(cudaStreamSynchronize(pl->last_stream));
  AWG_CUDA_TRY(cudaMemcpy(c, pl->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
  if (n_kept) *n_kept = (int64_t)c[0];
  if (n_dropped) *n_dropped = (int64_t)c[1];
  if (sum_taps) *sum_taps = (int64_t)c[2];
  return AWG_OK;
}

awg_status plan_copy_index(awg_plan h, int32_t* kept, int32_t* cf_out, int32_t* p0x, int32_t* p0y, int32_t* ox,
                           int32_t* oy) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "plan is NULL");
  PlanImpl* pl = (PlanImpl*)h;
  if (pl->n > 0 && (!kept || !cf_out || !p0x || !p0y || !ox || !oy))
    return set_error(AWG_ERR_INVALID_ARG, "output arrays must not be NULL");
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  AWG_CUDA_TRY(cudaStreamSynchronize(pl->last_stream));
  unsigned long long c[4];
  AWG_CUDA_TRY(cudaMemcpy(c, pl->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
  const int64_t n_kept_rec = (int64_t)c[0] * pl->rank;
  std::vector<SampleRec> rec;
  try {
    rec.resize((size_t)n_kept_rec);
  } catch (const std::bad_alloc&) {
    return set_error(AWG_ERR_OOM, "host allocation failed");
  }
  if (n_kept_rec > 0)
    AWG_CUDA_TRY(cudaMemcpy(rec.data(), pl->d_rec, sizeof(SampleRec) * (size_t)n_kept_rec, cudaMemcpyDeviceToHost));
  for (int64_t s = 0; s < pl->n; ++s) {
    kept[s] = 0;
    cf_out[s] = p0x[s] = p0y[s] = ox[s] = oy[s] = -1;
  }
  for (const SampleRec& r : rec) {
    if (r.src < 0 || r.src >= pl->n) return set_error(AWG_ERR_CUDA, "plan record outside the sample range");
    if (pl->rank > 1 && r.cf % pl->rank != 0) continue;   // term k > 0 of a sample: same index
    const int64_t s = r.src;
    kept[s] += 1;
    cf_out[s] = r.cf / pl->rank;
    p0x[s] = r.p0x;
    p0y[s] = r.p0y;
    ox[s] = r.ox;
    oy[s] = r.oy;
  }
  return AWG_OK;
}

awg_status plan_check(awg_plan h) {
  if (!h) return set_error(AWG_ERR_INVALID_ARG, "plan is NULL");
  PlanImpl* pl = (PlanImpl*)h;
  if (cudaSetDevice(pl->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  AWG_CUDA_TRY(cudaStreamSynchronize(pl->last_stream));
  unsigned long long c[4];
  AWG_CUDA_TRY(cudaMemcpy(c, pl->d_counters, sizeof(c), cudaMemcpyDeviceToHost));
  if (c[3] != 0) {
    const unsigned long long zero = 0;
    AWG_CUDA_TRY(cudaMemcpy(pl->d_counters + 3, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    return set_error(AWG_ERR_TIMEOUT, "a bounded wait of a gridding or degridding kernel gave up (its results are "
                                      "incomplete)");
  }
  return AWG_OK;
}

awg_status grid_visibilities(awg_cf_set hc, awg_plan hp, const void* vis, const float* weight, int32_t n_pol,
                             void* grid, void* grid_lo, double* sumwt, int32_t flags, void* stream) {
  NvtxRange nvtx_range("awg grid_visibilities");
  if (!hc || !hp) return set_error(AWG_ERR_INVALID_ARG, "cf set and plan must not be NULL");
  CfSetImpl* cf = (CfSetImpl*)hc;
  PlanImpl* pl = (PlanImpl*)hp;
  if (pl->cf != cf) return set_error(AWG_ERR_INVALID_ARG, "plan was made for another cf set");
  if (n_pol != 1 && n_pol != 2 && n_pol != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  if (flags & ~(AWG_GRID_KAHAN | AWG_GRID_FP64)) return set_error(AWG_ERR_INVALID_ARG, "unknown flags");
  if ((flags & AWG_GRID_KAHAN) && (flags & AWG_GRID_FP64))
    return set_error(AWG_ERR_INVALID_ARG, "AWG_GRID_KAHAN and AWG_GRID_FP64 are exclusive");
  if ((flags & AWG_GRID_KAHAN) && !grid_lo) return set_error(AWG_ERR_INVALID_ARG, "AWG_GRID_KAHAN needs grid_lo");
  if (pl->n > 0 && (!vis || !weight)) return set_error(AWG_ERR_INVALID_ARG, "vis and weight must not be NULL");
  if (!grid || !sumwt) return set_error(AWG_ERR_INVALID_ARG, "grid and sumwt must not be NULL");
  return launch_grid(cf, pl, vis, weight, n_pol, grid, grid_lo, sumwt, flags, (cudaStream_t)stream);
}

awg_status degrid_visibilities(awg_cf_set hc, awg_plan hp, const void* grid, void* vis_out, int32_t n_pol,
                               int32_t flags, void* stream) {
  NvtxRange nvtx_range("awg degrid_visibilities");
  if (!hc || !hp) return set_error(AWG_ERR_INVALID_ARG, "cf set and plan must not be NULL");
  CfSetImpl* cf = (CfSetImpl*)hc;
  PlanImpl* pl = (PlanImpl*)hp;
  if (pl->cf != cf) return set_error(AWG_ERR_INVALID_ARG, "plan was made for another cf set");
  if (n_pol != 1 && n_pol != 2 && n_pol != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  if ((flags & ~AWG_DEGRID_SUBTRACT) != 0)
    return set_error(AWG_ERR_INVALID_ARG, "degrid_visibilities flags: 0 or AWG_DEGRID_SUBTRACT");
  if (!grid || (pl->n > 0 && !vis_out)) return set_error(AWG_ERR_INVALID_ARG, "grid and vis_out must not be NULL");
  return launch_degrid(cf, pl, grid, vis_out, n_pol, (cudaStream_t)stream, (flags & AWG_DEGRID_SUBTRACT) != 0);
}

awg_status grid_normalize(awg_cf_set hc, void* image, int32_t n_pol, const double* sumwt, int32_t direction,
                          void* stream) {
  NvtxRange nvtx_range("awg grid_normalize");
  if (!hc || !image) return set_error(AWG_ERR_INVALID_ARG, "cf set and image must not be NULL");
  if (n_pol != 1 && n_pol != 2 && n_pol != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  if (direction != 0 && direction != 1) return set_error(AWG_ERR_INVALID_ARG, "direction must be 0 or 1");
  return launch_normalize((CfSetImpl*)hc, image, n_pol, sumwt, direction, (cudaStream_t)stream);
}

}  // extern "C"
