// Gridding and degridding with separable CFs, c[oy][ox][ty][tx] = fy[oy][ty] * fx[ox][tx].
//
// PS and W-projection CFs are outer products to FP32 precision (the W screen's non-separable
// part is below 1e-7 of the peak for fields of a fraction of a degree), so a sample needs only
// its two factor rows (2 S values) instead of an S x S slice.  A-term CFs are sums of a few such
// terms; the plan then holds one record per (sample, term), each a rank-1 sample of its own, so
// these kernels see only outer products.  The work decomposition is that of
// resample.cuh; the tap ownership is arranged so the factorisation also saves arithmetic:
//
// Thread t of NT owns column residue rx = t mod S and rows ry = t div S + k G, G = NT div S
// (threads t >= G S idle).  The window is pol-planar (tile[p][pixel]) so that the threads of a
// warp, which own consecutive columns, touch consecutive words.  Gridding: per sample the thread forms alpha_p = conj(fx[tx]) w V_p
// once for its column and then adds conj(fy[ty]) alpha_p for each of its rows: 4 FFMA per tap
// and pol, as with a full table, but the only per-tap load is fy[ty] from shared memory.
// Registers accumulate until a residue's pixel changes (column change: all rows; row change:
// that row); then they are added into the shared window, which is flushed with one vector
// atomic per pixel at the end of the item.
// Degridding: per sample the thread sums fy[ty] grid[Y][X][p] over its rows and multiplies by
// fx[tx] once; a warp reduce-scatter and a shared-memory pass finish the sum as in resample.cuh.
#pragma once

#include <type_traits>

#include "resample.cuh"

namespace awg {

// Row groups for support S on NT threads: G = NT / S (at most S); thread t < G S owns column
// t mod S and rows t div S + k G below S (the last rows of a column may be fewer).
__host__ __device__ constexpr int row_groups(int S, int nt) {
  int g = nt / S;
  if (g > S) g = S;
  return g < 1 ? 1 : g;
}

// Rows per thread needed by any support of a class: max over S in (smin, smax] of ceil(S / G).
__host__ __device__ constexpr int sep_rows(int smin, int smax, int nt) {
  int r = 1;
  for (int S = smin + 1; S <= smax; ++S) {
    const int g = row_groups(S, nt);
    const int rows = (S + g - 1) / g;
    r = rows > r ? rows : r;
  }
  return r;
}

// Staged samples per chunk of the class kernels: the factor rows of a chunk live in shared
// memory, twice (the chunk being computed and the one being fetched).
__host__ __device__ constexpr int sep_stage(int smax) { return smax >= 56 ? 8 : 16; }

// Shared-memory layout: the U x U window, then two slots of staged samples.  RK > 1 (fused
// kernels for CF sets of RK outer-product terms): a sample stages RK pairs of factor rows.
template <int SMAX, int TILE, int P, int ST, int RK = 1>
struct SepLayout {
  static constexpr int UMAX = TILE + SMAX - 1;
  // rounded up so that each slot starts 128-byte aligned (16-byte cp.async destinations)
  static constexpr size_t tile_bytes = ((size_t)UMAX * UMAX * P * sizeof(float2) + 127) & ~(size_t)127;
  // per slot
  static constexpr size_t f_off = 0;                                             // float2 [ST][2 RK][SMAX]
  static constexpr size_t v_off = f_off + (size_t)ST * 2 * RK * SMAX * sizeof(float2);  // float2 [ST][P]
  static constexpr size_t a_off = v_off + (size_t)ST * P * sizeof(float2);        // float2 [ST][P]
  static constexpr size_t w_off = a_off + (size_t)ST * P * sizeof(float2);        // float [ST][P] (padded)
  static constexpr size_t r_off = w_off + (((size_t)ST * P * sizeof(float) + 15) & ~(size_t)15);  // SampleRec [ST]
  static constexpr size_t x_off = r_off + (size_t)ST * sizeof(SampleRec);          // long long [ST][RK] fx offsets
  static constexpr size_t y_off = x_off + (size_t)ST * RK * sizeof(long long);     // long long [ST][RK] fy offsets
  static constexpr size_t ph_off = y_off + (size_t)ST * RK * sizeof(long long);    // float2 [ST]
  static constexpr size_t k_off = ph_off + (size_t)ST * sizeof(float2);            // int [ST] packed offsets
  static constexpr size_t s_off = k_off + (size_t)ST * sizeof(int);                // int [ST] sample index
  static constexpr size_t slot_bytes = (s_off + (size_t)ST * sizeof(int) + 127) & ~(size_t)127;
  // per-chunk table by column residue: gridding alpha[j][rx][p] = conj(fx[j][tx]) w V_p,
  // degridding beta[j][rx] = fx[j][tx], tx = (rx - p0x) mod S; with RK > 1 both hold the terms
  // beta[j][rx][t] = fx_t[j][tx] (conjugated for gridding)
  static constexpr size_t al_off = tile_bytes + 2 * slot_bytes;
  static constexpr size_t al_bytes = (size_t)ST * SMAX * (RK > 1 ? RK : P) * sizeof(float2);
  static constexpr size_t bytes = al_off + al_bytes;
};

// CTAs per SM that the shared-memory window allows (228 KB per SM, 1 KB reserved per CTA),
// capped so that each thread keeps at least min_regs registers (96; 128 for the fused kernels,
// which also hold the CF terms and w V): the min-blocks hint of the kernels.
__host__ __device__ constexpr int sep_min_blocks(size_t smem_bytes, int nt, int min_regs = 96) {
  const int by_smem = (int)(233472 / (smem_bytes + 1024));
  const int by_regs = 65536 / (nt * min_regs);
  const int b = by_smem < by_regs ? by_smem : by_regs;
  return b < 1 ? 1 : b;
}

template <int SMAX, int TILE, int P, int ST, int RK = 1>
struct SepSlot {
  using L = SepLayout<SMAX, TILE, P, ST, RK>;
  unsigned char* base;
  __device__ SepSlot(unsigned char* smem, int slot) : base(smem + L::tile_bytes + slot * L::slot_bytes) {}
  __device__ float2* f() const { return reinterpret_cast<float2*>(base + L::f_off); }
  __device__ float2* v() const { return reinterpret_cast<float2*>(base + L::v_off); }
  __device__ float2* a() const { return reinterpret_cast<float2*>(base + L::a_off); }
  __device__ float* w() const { return reinterpret_cast<float*>(base + L::w_off); }
  __device__ SampleRec* rec() const { return reinterpret_cast<SampleRec*>(base + L::r_off); }
  __device__ long long* fxo() const { return reinterpret_cast<long long*>(base + L::x_off); }
  __device__ long long* fyo() const { return reinterpret_cast<long long*>(base + L::y_off); }
  __device__ float2* ph() const { return reinterpret_cast<float2*>(base + L::ph_off); }
  __device__ int* pack() const { return reinterpret_cast<int*>(base + L::k_off); }
  __device__ int* src() const { return reinterpret_cast<int*>(base + L::s_off); }
};

__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src));
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Records of chunk c into a slot (threads < nst, one 16-byte copy each).
template <int SMAX, int TILE, int P, int ST, int RK>
__device__ __forceinline__ void stage_recs(const SampleRec* rec, int start, int nst,
                                           const SepSlot<SMAX, TILE, P, ST, RK>& sl) {
  if ((int)threadIdx.x < nst) cp_async(sl.rec() + threadIdx.x, rec + start + threadIdx.x, 16);
}

// Factor offsets the rank-1 kernels keep in shared memory when the whole table fits (one entry
// per CF and term: 127 for the W-projection set of 64 planes).
constexpr int kSepOffCache = 256;

// From staged records: packed window offsets, factor-row offsets, sample index, phasor.  `offs` is
// the factor-offset table (a.sep_off, or its copy in shared memory).
template <int SMAX, int TILE, int P, int ST, int RK, class Args>
__device__ __forceinline__ void derive(const Args& a, const int64_t* offs, int nst, int S, int X0, int Y0,
                                       const SepSlot<SMAX, TILE, P, ST, RK>& sl) {
  const int j = threadIdx.x;
  if (j < nst) {
    const SampleRec rc = sl.rec()[j];
    // RK == 1: the record's own term; RK > 1: the CF's RK terms at sep_off[cf RK + t]
#pragma unroll
    for (int t = 0; t < RK; ++t) {
      const long long base = offs[a.cf_shift + (RK == 1 ? rc.cf : rc.cf * RK + t)];
      sl.fxo()[j * RK + t] = base + (long long)rc.ox * S;
      sl.fyo()[j * RK + t] = base + (long long)(a.OS + 1) * S + (long long)rc.oy * S;
    }
    sl.pack()[j] = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | ((rc.p0x % S) << 16) | ((rc.p0y % S) << 24);
    if constexpr (std::is_same<Args, DegridArgs>::value)   // the output row of this record
      sl.src()[j] = a.rank > 1 ? rc.src * a.rank + rc.cf % a.rank : rc.src;
    else   // the visibility / weight row
      sl.src()[j] = rc.src;
    sl.ph()[j] = a.phasor ? a.phasor[rc.src] : make_float2(1.f, 0.f);
  }
}

// Asynchronous copies of a chunk's factor rows (all threads) and, when vis != NULL, its
// visibilities and weights (threads < nst).
template <int SMAX, int TILE, int P, int ST, int NT, int RK>
__device__ __forceinline__ void stage_payload(const float* sep, const float* vis, const float* weight, int nst, int S,
                                              const SepSlot<SMAX, TILE, P, ST, RK>& sl, int vstride = P,
                                              int voff = 0) {
  const float2* sep2 = reinterpret_cast<const float2*>(sep);
  const long long* fxo = sl.fxo();
  const long long* fyo = sl.fyo();
  float2* f = sl.f();
  // row 2 t of sample j holds fx of term t, row 2 t + 1 its fy
  for (int i = threadIdx.x; i < nst * 2 * RK * S; i += NT) {
    const int jt = i / (2 * S), r = i - jt * 2 * S;   // jt = j RK + t
    const bool isx = r < S;
    const long long srcidx = isx ? fxo[jt] + r : fyo[jt] + (r - S);
    cp_async(f + (jt * 2 + (isx ? 0 : 1)) * SMAX + (isx ? r : r - S), sep2 + srcidx, 8);
  }
  if (vis != nullptr && (int)threadIdx.x < nst) {
    const int j = threadIdx.x;
    const size_t s = (size_t)sl.src()[j];
    const float* vp = vis + (s * vstride + voff) * 2;
    const float* wp = weight + s * vstride + voff;
    if (P == 4) {
      cp_async(sl.v() + j * P, vp, 16);
      cp_async(sl.v() + j * P + 2, vp + 4, 16);
      cp_async(sl.w() + j * P, wp, 16);
    } else if (P == 2) {
      cp_async(sl.v() + j * P, vp, 16);
      cp_async(sl.w() + j * P, wp, 8);
    } else {
      cp_async(sl.v() + j * P, vp, 8);
      cp_async(sl.w() + j * P, wp, 4);
    }
  }
}

// Column residue rx and first row ry0 of thread t (it owns rows ry0 + k G).  Generic: rx = t mod S,
// ry0 = t div S.  For an exact support that is a multiple of 8 whose warps tile the columns in
// blocks of 8 (NT / 32 a multiple of S / 8), a warp instead covers 8 consecutive columns x 4 row
// groups: its per-sample column loads (alpha, beta) then touch 8 distinct addresses, one
// shared-memory wavefront, instead of 32.  Both mappings give every (column, row group) pair to
// exactly one thread.  Degridding without the register grid cache reads the window for every
// tap, where 4 rows per warp cost bank conflicts; it keeps the generic mapping.
template <int SMIN, int SMAX, int NT, bool BLOCKED_OK>
__device__ __forceinline__ void tap_owner(int t, int S, int& rx, int& ry0) {
  constexpr bool kBlocked = BLOCKED_OK && SMIN + 1 == SMAX && SMAX % 8 == 0 && (NT / 32) % (SMAX / 8) == 0;
  if constexpr (kBlocked) {
    constexpr int kColBlocks = SMAX / 8;
    const int lane = t & 31, w = t >> 5;
    rx = (w % kColBlocks) * 8 + (lane & 7);
    ry0 = (w / kColBlocks) * 4 + (lane >> 3);
  } else {
    rx = t % S;
    ry0 = t / S;
  }
}

// P consecutive complex values from shared memory (16-byte loads where the layout allows).
template <int P>
__device__ __forceinline__ void load_pols(const float2* src, float2 (&out)[P]) {
  if constexpr (P % 2 == 0) {
#pragma unroll
    for (int q = 0; q < P / 2; ++q) {
      const float4 v = reinterpret_cast<const float4*>(src)[q];
      out[2 * q] = make_float2(v.x, v.y);
      out[2 * q + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) out[p] = src[p];
  }
}

// Per-thread row state of the separable kernels.  The rows a thread owns are ry0 + k G (k < R,
// valid while below S); for a sample whose first tap is (p0x, p0y) the row residue ry touches
// window row dy + ((ry - p0y) mod S).  Samples of an item are sorted row-major, so that state is
// recomputed only when p0y changes (a test that is uniform across the CTA).
template <int R>
struct RowState {
  int ty[R];   // tap row of each owned row for the current p0y
  int Y[R];    // window row of each owned row for the current p0y
  __device__ __forceinline__ void update(int ry0, int G, int S, int dy, int my, unsigned vmask) {
    int ty0 = ry0 - my;
    ty0 += (ty0 < 0) ? S : 0;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (vmask & (1u << k)) {
        int t = ty0 + k * G;
        t -= (t >= S) ? S : 0;
        ty[k] = t;
        Y[k] = dy + t;
      }
    }
  }
};

// u_q = sum_p mix[4 q + p] w_p V_p for the 4 pols of one staged sample (full-polarisation base
// launches).
__device__ __forceinline__ void mix_pols(const float2* __restrict__ mix, const float2* v, const float* w,
                                         float2 (&u)[4]) {
  float2 wv[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) wv[p] = make_float2(w[p] * v[p].x, w[p] * v[p].y);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float2 m = __ldg(mix + 4 * q + p);
      acc.x = fmaf(m.x, wv[p].x, fmaf(-m.y, wv[p].y, acc.x));
      acc.y = fmaf(m.x, wv[p].y, fmaf(m.y, wv[p].x, acc.y));
    }
    u[q] = acc;
  }
}

// alpha[j][rx][p] = conj(fx[j][(rx - mx_j) mod S]) * w_jp V_jp (* phasor): formed once per
// chunk for every (sample, column residue) instead of by each of the G threads of a column.  The
// threads below nst also add the chunk's weights to the sum of weights (term 0 of each sample).
// The MIX instances of the fused kernels (P = 4) serve the base passes of full-polarisation sets:
// only the pols in pmask add weights, and the mixed u_q of mix_pols take the place of w V.
template <int SMAX, int TILE, int P, int ST, int NT, int RK, bool MIX>
__device__ __forceinline__ void form_alpha(const SepSlot<SMAX, TILE, P, ST, RK>& sl, float2* alpha, int nst, int S,
                                           int rank, double (&wsum)[P], const float2* mix, int pmask) {
  static_assert(!MIX || (P == 4 && RK > 1), "pol mixing is compiled into the 4-pol fused kernels only");
  if ((int)threadIdx.x < nst && (rank == 1 || sl.rec()[threadIdx.x].cf % rank == 0)) {
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (!MIX || ((pmask >> p) & 1)) wsum[p] += (double)sl.w()[threadIdx.x * P + p];
  }
  if constexpr (RK > 1) {
    // fused terms: w V (* phasor) per sample into the slot's a(), conj(fx_t) per column residue
    if ((int)threadIdx.x < nst) {
      const int j = threadIdx.x;
      const float2 ph = sl.ph()[j];
      if constexpr (MIX) {
        float2 u[4];
        mix_pols(mix, sl.v() + j * 4, sl.w() + j * 4, u);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          sl.a()[j * 4 + q] = make_float2(u[q].x * ph.x - u[q].y * ph.y, u[q].x * ph.y + u[q].y * ph.x);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float wv = sl.w()[j * P + p];
          const float2 v = sl.v()[j * P + p];
          const float xr = wv * v.x, xi = wv * v.y;
          sl.a()[j * P + p] = make_float2(xr * ph.x - xi * ph.y, xr * ph.y + xi * ph.x);
        }
      }
    }
    for (int i = threadIdx.x; i < nst * S; i += NT) {
      const int j = i / S, rx = i - j * S;
      const int mx = (sl.pack()[j] >> 16) & 0xff;
      int tx = rx - mx;
      tx += (tx < 0) ? S : 0;
#pragma unroll
      for (int t = 0; t < RK; ++t) {
        const float2 fxv = sl.f()[(j * 2 * RK + 2 * t) * SMAX + tx];
        alpha[(j * SMAX + rx) * RK + t] = make_float2(fxv.x, -fxv.y);
      }
    }
    return;
  }
  for (int i = threadIdx.x; i < nst * S; i += NT) {
    const int j = i / S, rx = i - j * S;
    const int mx = (sl.pack()[j] >> 16) & 0xff;
    int tx = rx - mx;
    tx += (tx < 0) ? S : 0;
    const float2 fxv = sl.f()[(j * 2) * SMAX + tx];
    const float2 ph = sl.ph()[j];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float wv = sl.w()[j * P + p];
      const float2 v = sl.v()[j * P + p];
      const float xr = wv * v.x, xi = wv * v.y;
      const float ar = xr * ph.x - xi * ph.y, ai = xr * ph.y + xi * ph.x;
      alpha[(j * SMAX + rx) * P + p] = make_float2(fxv.x * ar + fxv.y * ai, fxv.x * ai - fxv.y * ar);
    }
  }
}

// beta[j][rx] = fx[j][(rx - mx_j) mod S] for the degridding kernel.
template <int SMAX, int TILE, int P, int ST, int NT, int RK>
__device__ __forceinline__ void form_beta(const SepSlot<SMAX, TILE, P, ST, RK>& sl, float2* beta, int nst, int S) {
  for (int i = threadIdx.x; i < nst * S; i += NT) {
    const int j = i / S, rx = i - j * S;
    const int mx = (sl.pack()[j] >> 16) & 0xff;
    int tx = rx - mx;
    tx += (tx < 0) ? S : 0;
#pragma unroll
    for (int t = 0; t < RK; ++t) beta[(j * SMAX + rx) * RK + t] = sl.f()[(j * 2 * RK + 2 * t) * SMAX + tx];
  }
}

template <int SMIN, int SMAX, int NT, int TILE, int P, int ST, int RK = 1, bool MIX = false>
__global__ void __launch_bounds__(NT, sep_min_blocks(SepLayout<SMAX, TILE, P, ST, RK>::bytes, NT, RK > 1 ? 128 : 96))
    k_grid_sep(const GridArgs a, const int cls) {
  constexpr int R = sep_rows(SMIN, SMAX, NT);
  using Slot = SepSlot<SMAX, TILE, P, ST, RK>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float2* alpha = reinterpret_cast<float2*>(smem + SepLayout<SMAX, TILE, P, ST, RK>::al_off);
  __shared__ int s_item;
  __shared__ double s_wsum[NT / 32][P];
  __shared__ int64_t s_off[RK == 1 ? kSepOffCache : 1];
  static_assert(NT % 32 == 0, "the warp reductions need whole warps");

  const int tid = threadIdx.x;
  const int begin = a.class_range[cls], end = a.class_range[cls + 1];
  // a small factor-offset table is read from shared memory (visible after the item loop's first
  // barrier), so that derive() makes no global round trip while the other warps wait
  if (RK == 1 && a.n_sep_off <= kSepOffCache)
    for (int i = tid; i < a.n_sep_off; i += NT) s_off[i] = a.sep_off[i];
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
    const int S = (SMIN + 1 == SMAX) ? SMAX : (int)wi.S;   // a constant for exact-support kernels
    const int U = TILE + S - 1;
    const int X0 = wi.tile_x * TILE, Y0 = wi.tile_y * TILE;
    const int G = row_groups(S, NT);
    const bool active = tid < G * S;
    int rx, ry0;
    tap_owner<SMIN, SMAX, NT, true>(tid, S, rx, ry0);
    unsigned vmask = 0;
#pragma unroll
    for (int k = 0; k < R; ++k) vmask |= (ry0 + k * G < S) ? (1u << k) : 0u;
    if (SMIN + 1 == SMAX) vmask = (1u << R) - 1;   // G divides S: every thread owns R rows
    const int nch = (wi.count + ST - 1) / ST;
    auto nst_of = [&](int c) { return min(ST, wi.count - c * ST); };
    const int UU = U * U;   // the window is pol-planar: tile[p * UU + pixel]
    for (int i = tid; i < UU * P; i += NT) tile[i] = make_float2(0.f, 0.f);
    // prologue: records of chunks 0 and 1, derived data of chunks 0 and 1, payload of chunk 0
    {
      const Slot s0(smem, 0), s1(smem, 1);
      stage_recs(a.rec, wi.start, nst_of(0), s0);
      if (nch > 1) stage_recs(a.rec, wi.start + ST, nst_of(1), s1);
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      derive(a, RK == 1 && a.n_sep_off <= kSepOffCache ? s_off : a.sep_off, nst_of(0), S, X0, Y0, s0);
      if (nch > 1) derive(a, RK == 1 && a.n_sep_off <= kSepOffCache ? s_off : a.sep_off, nst_of(1), S, X0, Y0, s1);
      __syncthreads();
      stage_payload<SMAX, TILE, P, ST, NT, RK>(a.sep, a.vis, a.weight, nst_of(0), S, s0, a.vstride, a.voff);
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      form_alpha<SMAX, TILE, P, ST, NT, RK, MIX>(s0, alpha, nst_of(0), S, a.rank, wsum, a.mix, a.pmask);
      __syncthreads();
    }

    RowState<R> rs;
    int prev_row = -1, prev_pk = -1;
    int curX = -1;
    int curY[R];
    float2 acc[R][P];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      curY[k] = -1;
      rs.ty[k] = 0;
      rs.Y[k] = -1;
#pragma unroll
      for (int p = 0; p < P; ++p) acc[k][p] = make_float2(0.f, 0.f);
    }
    for (int c = 0; c < nch; ++c) {
      const Slot A(smem, c & 1), B(smem, (c & 1) ^ 1);
      if (c + 1 < nch) stage_payload<SMAX, TILE, P, ST, NT, RK>(a.sep, a.vis, a.weight, nst_of(c + 1), S, B, a.vstride, a.voff);
      if (c + 2 < nch) stage_recs(a.rec, wi.start + (c + 2) * ST, nst_of(c + 2), A);
      cp_async_commit();
      const int nst = nst_of(c);
      if (active) {
        for (int j = 0; j < nst; ++j) {
          const int pk = A.pack()[j];
          // RK == 1: al = alpha_p = conj(fx) w V_p; RK > 1: bt_t = conj(fx_t), wv_p = w V_p
          float2 al[RK > 1 ? RK : P];
          float2 wv[P];
          if constexpr (RK == 1) {
            load_pols<P>(alpha + (j * SMAX + rx) * P, al);
          } else {
            load_pols<RK>(alpha + (j * SMAX + rx) * RK, al);
            load_pols<P>(A.a() + j * P, wv);
          }
          if (pk != prev_pk) {   // the first tap moved (the same test in every thread of the CTA)
            prev_pk = pk;
            const int dx = pk & 0xff, mx = (pk >> 16) & 0xff;
            const int row = pk & 0xff00ff00;   // (dy, my)
            bool row_changed = false;
            if (row != prev_row) {
              prev_row = row;
              rs.update(ry0, G, S, (pk >> 8) & 0xff, (pk >> 24) & 0xff, vmask);
              row_changed = true;
            }
            int tx = rx - mx;
            tx += (tx < 0) ? S : 0;
            const int X = dx + tx;
            if (X != curX || row_changed) {
              const bool xchg = X != curX;
#pragma unroll
              for (int k = 0; k < R; ++k) {
                if ((vmask & (1u << k)) && (xchg || rs.Y[k] != curY[k])) {
                  if (curY[k] >= 0) {
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                      float2* t = tile + p * UU + curY[k] * U + curX;
                      t->x += acc[k][p].x;
                      t->y += acc[k][p].y;
                      acc[k][p] = make_float2(0.f, 0.f);
                    }
                  }
                  curY[k] = rs.Y[k];
                }
              }
              curX = X;
            }
          }
          if constexpr (RK == 1) {
            const float2* fyrow = A.f() + (j * 2 + 1) * SMAX;
#pragma unroll
            for (int k = 0; k < R; ++k) {
              if (vmask & (1u << k)) {
                const float2 f = fyrow[rs.ty[k]];
#pragma unroll
                for (int p = 0; p < P; ++p) {   // acc += conj(fy) alpha
                  acc[k][p].x = fmaf(f.x, al[p].x, fmaf(f.y, al[p].y, acc[k][p].x));
                  acc[k][p].y = fmaf(f.x, al[p].y, fmaf(-f.y, al[p].x, acc[k][p].y));
                }
              }
            }
          } else {
            const float2* frows = A.f() + (j * 2 * RK + 1) * SMAX;   // fy of term t at 2 t SMAX further
#pragma unroll
            for (int k = 0; k < R; ++k) {
              if (vmask & (1u << k)) {
                // c = conj(CF) at this tap = sum_t conj(fy_t) conj(fx_t)
                float2 c = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < RK; ++t) {
                  const float2 f = frows[2 * t * SMAX + rs.ty[k]];
                  c.x = fmaf(f.x, al[t].x, fmaf(f.y, al[t].y, c.x));
                  c.y = fmaf(f.x, al[t].y, fmaf(-f.y, al[t].x, c.y));
                }
#pragma unroll
                for (int p = 0; p < P; ++p) {   // acc += c w V_p
                  acc[k][p].x = fmaf(c.x, wv[p].x, fmaf(-c.y, wv[p].y, acc[k][p].x));
                  acc[k][p].y = fmaf(c.x, wv[p].y, fmaf(c.y, wv[p].x, acc[k][p].y));
                }
              }
            }
          }
        }
      }
      cp_async_wait_all();
      __syncthreads();
      // slot A is free: derive chunk c+2 into it; chunk c+1's payload has landed in B: form w V
      if (c + 2 < nch) derive(a, RK == 1 && a.n_sep_off <= kSepOffCache ? s_off : a.sep_off, nst_of(c + 2), S, X0, Y0, A);
      if (c + 1 < nch) form_alpha<SMAX, TILE, P, ST, NT, RK, MIX>(B, alpha, nst_of(c + 1), S, a.rank, wsum, a.mix, a.pmask);
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      if (curY[k] >= 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          float2* t = tile + p * UU + curY[k] * U + curX;
          t->x += acc[k][p].x;
          t->y += acc[k][p].y;
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < UU; i += NT) {
      const int ly = i / U, lx = i - ly * U;
      const int gy = Y0 + ly, gx = X0 + lx;
      if (gy >= a.N || gx >= a.N) continue;
      float2 v[P];
      bool nz = false;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        v[p] = tile[p * UU + i];
        nz |= (v[p].x != 0.f) || (v[p].y != 0.f);
      }
      if (nz) flush_pixel<P>(a, ((size_t)gy * a.N + gx) * a.gstride + a.goff, v);
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
  if (tid < P && a.sumwt) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += s_wsum[w][tid];
    if (v != 0.0) atomicAdd(a.sumwt + tid, v);
  }
}

// Degridding keeps the window pixels of its rows in registers (reloaded when a pixel changes)
// when they fit; otherwise it reads them from the pol-planar window for every sample.
template <int R, int P>
struct DegridCache {
  static constexpr bool enabled = R * P * 2 <= 48;
};

template <int SMIN, int SMAX, int NT, int TILE, int P, int ST, int RK = 1, bool MIX = false>
__global__ void __launch_bounds__(NT, sep_min_blocks(SepLayout<SMAX, TILE, P, ST, RK>::bytes, NT, RK > 1 ? 128 : 96))
    k_degrid_sep(const DegridArgs a, const int cls) {
  constexpr int R = sep_rows(SMIN, SMAX, NT);
  constexpr int NW = NT / 32;
  static_assert(NT % 32 == 0, "the warp reductions need whole warps");
  constexpr int B = 32 / (2 * P);
  constexpr bool CACHE = DegridCache<R, P>::enabled;
  constexpr int RC = CACHE ? R : 1;
  using Slot = SepSlot<SMAX, TILE, P, ST, RK>;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tile = reinterpret_cast<float2*>(smem);
  float2* beta = reinterpret_cast<float2*>(smem + SepLayout<SMAX, TILE, P, ST, RK>::al_off);
  // per-warp butterfly results of every batch of the chunk; combined once per chunk
  constexpr int NB = (ST + B - 1) / B;          // batches per chunk
  constexpr int NBW = (NB + NW - 1) / NW;       // batches combined by one warp
  __shared__ float s_red[NB][NW][32];
  __shared__ int s_item;
  __shared__ int64_t s_off[RK == 1 ? kSepOffCache : 1];

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int begin = a.class_range[cls], end = a.class_range[cls + 1];
  // a small factor-offset table is read from shared memory (as in k_grid_sep)
  if (RK == 1 && a.n_sep_off <= kSepOffCache)
    for (int i = tid; i < a.n_sep_off; i += NT) s_off[i] = a.sep_off[i];

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = begin + atomicAdd(a.queue + cls, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= end) break;
    const WorkItem wi = a.items[it];
    const int S = (SMIN + 1 == SMAX) ? SMAX : (int)wi.S;   // a constant for exact-support kernels
    const int U = TILE + S - 1;
    const int X0 = wi.tile_x * TILE, Y0 = wi.tile_y * TILE;
    const int G = row_groups(S, NT);
    const bool active = tid < G * S;
    int rx, ry0;
    tap_owner<SMIN, SMAX, NT, CACHE>(tid, S, rx, ry0);
    unsigned vmask = 0;
#pragma unroll
    for (int k = 0; k < R; ++k) vmask |= (ry0 + k * G < S) ? (1u << k) : 0u;
    if (SMIN + 1 == SMAX) vmask = (1u << R) - 1;   // G divides S: every thread owns R rows
    const int nch = (wi.count + ST - 1) / ST;
    auto nst_of = [&](int c) { return min(ST, wi.count - c * ST); };
    const int UU = U * U;   // the window is pol-planar: tile[p * UU + pixel]
    {
      const Slot s0(smem, 0), s1(smem, 1);
      stage_recs(a.rec, wi.start, nst_of(0), s0);
      if (nch > 1) stage_recs(a.rec, wi.start + ST, nst_of(1), s1);
      cp_async_commit();
      // the window: asynchronous 8-byte copies of the on-grid pixels (in flight together with the
      // records instead of one dependent load and store after another), zeros off the grid
      for (int i = tid; i < UU; i += NT) {
        const int ly = i / U, lx = i - ly * U;
        const int gy = Y0 + ly, gx = X0 + lx;
        if (gy < a.N && gx < a.N) {
          const float2* src = reinterpret_cast<const float2*>(a.grid) + ((size_t)gy * a.N + gx) * a.gstride + a.goff;
#pragma unroll
          for (int p = 0; p < P; ++p) cp_async(tile + p * UU + i, src + p, 8);
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p) tile[p * UU + i] = make_float2(0.f, 0.f);
        }
      }
      cp_async_wait_all();
      __syncthreads();
      derive(a, RK == 1 && a.n_sep_off <= kSepOffCache ? s_off : a.sep_off, nst_of(0), S, X0, Y0, s0);
      if (nch > 1) derive(a, RK == 1 && a.n_sep_off <= kSepOffCache ? s_off : a.sep_off, nst_of(1), S, X0, Y0, s1);
      __syncthreads();
      stage_payload<SMAX, TILE, P, ST, NT, RK>(a.sep, nullptr, nullptr, nst_of(0), S, s0);
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      form_beta<SMAX, TILE, P, ST, NT, RK>(s0, beta, nst_of(0), S);
      __syncthreads();
    }
    RowState<R> rs;
    int prev_row = -1, prev_pk = -1;
    int curX = -1, X = 0;
    int curY[RC];
    float2 gc[RC][P];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      rs.ty[k] = 0;
      rs.Y[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < RC; ++k) curY[k] = -1;
    for (int c = 0; c < nch; ++c) {
      const Slot A(smem, c & 1), Bs(smem, (c & 1) ^ 1);
      if (c + 1 < nch) stage_payload<SMAX, TILE, P, ST, NT, RK>(a.sep, nullptr, nullptr, nst_of(c + 1), S, Bs);
      if (c + 2 < nch) stage_recs(a.rec, wi.start + (c + 2) * ST, nst_of(c + 2), A);
      cp_async_commit();
      const int nst = nst_of(c);
      int cap_src[NBW];
      float2 cap_ph[NBW];
#pragma unroll
      for (int q = 0; q < NBW; ++q) cap_src[q] = -1;
      for (int j0 = 0; j0 < nst; j0 += B) {
        float vals[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) vals[q] = 0.f;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int j = j0 + b;
          if (active && j < nst) {
            const int pk = A.pack()[j];
            // RK == 1: fxv = fx[tx] applied after the rows; RK > 1: bt_t = fx_t[tx] inside each row
            float2 bt[RK];
            if constexpr (RK == 1) bt[0] = beta[j * SMAX + rx];
            else load_pols<RK>(beta + (j * SMAX + rx) * RK, bt);
            const float2 fxv = RK == 1 ? bt[0] : make_float2(1.f, 0.f);
            if (pk != prev_pk) {   // the first tap moved (the same test in every thread of the CTA)
              prev_pk = pk;
              const int dx = pk & 0xff, mx = (pk >> 16) & 0xff;
              const int row = pk & 0xff00ff00;
              bool row_changed = false;
              if (row != prev_row) {
                prev_row = row;
                rs.update(ry0, G, S, (pk >> 8) & 0xff, (pk >> 24) & 0xff, vmask);
                row_changed = true;
              }
              int tx = rx - mx;
              tx += (tx < 0) ? S : 0;
              X = dx + tx;
              if constexpr (CACHE) {
                if (X != curX || row_changed) {
                  const bool xchg = X != curX;
#pragma unroll
                  for (int k = 0; k < RC; ++k) {
                    if ((vmask & (1u << k)) && (xchg || rs.Y[k] != curY[k])) {
                      curY[k] = rs.Y[k];
#pragma unroll
                      for (int p = 0; p < P; ++p) gc[k][p] = tile[p * UU + curY[k] * U + X];
                    }
                  }
                  curX = X;
                }
              }
            }
            const float2* fyrow = A.f() + (j * 2 * RK + 1) * SMAX;   // fy of term t at 2 t SMAX further
            float2 part[P];
#pragma unroll
            for (int p = 0; p < P; ++p) part[p] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < R; ++k) {
              if (vmask & (1u << k)) {
                float2 f;
                if constexpr (RK == 1) {
                  f = fyrow[rs.ty[k]];
                } else {   // the CF at this tap: sum_t fy_t fx_t
                  f = make_float2(0.f, 0.f);
#pragma unroll
                  for (int t = 0; t < RK; ++t) {
                    const float2 y = fyrow[2 * t * SMAX + rs.ty[k]];
                    f.x = fmaf(y.x, bt[t].x, fmaf(-y.y, bt[t].y, f.x));
                    f.y = fmaf(y.x, bt[t].y, fmaf(y.y, bt[t].x, f.y));
                  }
                }
#pragma unroll
                for (int p = 0; p < P; ++p) {
                  float2 gv;
                  if constexpr (CACHE) gv = gc[k < RC ? k : 0][p];
                  else gv = tile[p * UU + rs.Y[k] * U + X];
                  part[p].x = fmaf(f.x, gv.x, fmaf(-f.y, gv.y, part[p].x));
                  part[p].y = fmaf(f.x, gv.y, fmaf(f.y, gv.x, part[p].y));
                }
              }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
              if constexpr (RK == 1) {
                vals[b * 2 * P + 2 * p] = fxv.x * part[p].x - fxv.y * part[p].y;
                vals[b * 2 * P + 2 * p + 1] = fxv.x * part[p].y + fxv.y * part[p].x;
              } else {
                vals[b * 2 * P + 2 * p] = part[p].x;
                vals[b * 2 * P + 2 * p + 1] = part[p].y;
              }
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
        const int bi = j0 / B;
        s_red[bi][wid][lane] = vals[0];
        if (bi % NW == wid) {   // this warp combines the batch: keep its output rows and phasors
          const int j = j0 + lane / (2 * P);
          const int src = j < nst ? A.src()[j] : -1;
          const float2 ph = j < nst ? A.ph()[j] : make_float2(1.f, 0.f);
          if constexpr (NBW == 1) {
            cap_src[0] = src;
            cap_ph[0] = ph;
          } else {
#pragma unroll
            for (int q = 0; q < NBW; ++q)   // static indices keep the arrays in registers
              if (q == bi / NW) {
                cap_src[q] = src;
                cap_ph[q] = ph;
              }
          }
        }
      }
      cp_async_wait_all();
      __syncthreads();
      {
        // warp w adds up the warps' partials of batches w, w + NW, ... and writes whole samples
        const int nbat = (nst + B - 1) / B;
        const int comp = lane - (lane / (2 * P)) * 2 * P;
#pragma unroll
        for (int q = 0; q < NBW; ++q) {
          const int bi = wid + q * NW;
          if (bi < nbat) {
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) v += s_red[bi][w][lane];
            const float partner = __shfl_xor_sync(0xffffffffu, v, 1);
            if constexpr (!MIX) {
              if (cap_src[q] >= 0) {
                const float2 ph = cap_ph[q];
                const float out = (comp & 1) ? (v * ph.x - partner * ph.y) : (v * ph.x + partner * ph.y);
                float* o = a.vis_out + ((size_t)cap_src[q] * a.vstride + a.voff) * 2 + comp;
                *o = a.accumulate == 0 ? out : a.accumulate > 0 ? *o + out : *o - out;
              }
            } else {
              const float2 ph = cap_ph[q];
              float out = (comp & 1) ? (v * ph.x - partner * ph.y) : (v * ph.x + partner * ph.y);
              static_assert(!MIX || (P == 4 && RK > 1), "pol mixing is compiled into the 4-pol fused kernels only");
              {
                // the sample's 8 lanes hold Y_0..Y_3 (re, im): output pol p = sum_q mix[4 p + q] Y_q
                const float other = __shfl_xor_sync(0xffffffffu, out, 1);
                const float yr = (comp & 1) ? other : out, yi = (comp & 1) ? out : other;
                const int base = lane & ~7, p = comp >> 1;
                float ar = 0.f, ai = 0.f;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                  const float2 m = __ldg(a.mix + 4 * p + qq);
                  const float zr = __shfl_sync(0xffffffffu, yr, base + 2 * qq);
                  const float zi = __shfl_sync(0xffffffffu, yi, base + 2 * qq);
                  ar = fmaf(m.x, zr, fmaf(-m.y, zi, ar));
                  ai = fmaf(m.x, zi, fmaf(m.y, zr, ai));
                }
                out = (comp & 1) ? ai : ar;
              }
              if (cap_src[q] >= 0 && ((a.pmask >> (comp >> 1)) & 1)) {
                float* o = a.vis_out + ((size_t)cap_src[q] * a.vstride + a.voff) * 2 + comp;
                *o = a.accumulate == 0 ? out : a.accumulate > 0 ? *o + out : *o - out;
              }
            }
          }
        }
      }
      if (c + 2 < nch) derive(a, RK == 1 && a.n_sep_off <= kSepOffCache ? s_off : a.sep_off, nst_of(c + 2), S, X0, Y0, A);
      if (c + 1 < nch) form_beta<SMAX, TILE, P, ST, NT, RK>(Bs, beta, nst_of(c + 1), S);
      __syncthreads();
    }
  }
}

// Threads per CTA of the separable kernels by class: enough warps per SM to hide latency while
// each thread keeps several rows of its column in registers.
constexpr int kSepThreads[kNumClasses] = {128, 256, 256, 512, 512, 512};

template <int CLS, int P>
awg_status run_grid_sep(const GridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr ClassCfg cc = kClasses[CLS];
  constexpr int smin = CLS == 0 ? 0 : kClasses[CLS > 0 ? CLS - 1 : 0].smax;
  constexpr int nt = kSepThreads[CLS];
  constexpr int st_depth = sep_stage(cc.smax);
  using L = SepLayout<cc.smax, cc.tile, P, st_depth>;
  auto kern = k_grid_sep<smin, cc.smax, nt, cc.tile, P, st_depth>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cc.nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "separable gridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, nt, L::bytes, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

template <int CLS, int P>
awg_status run_degrid_sep(const DegridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr ClassCfg cc = kClasses[CLS];
  constexpr int smin = CLS == 0 ? 0 : kClasses[CLS > 0 ? CLS - 1 : 0].smax;
  constexpr int nt = kSepThreads[CLS];
  constexpr int st_depth = sep_stage(cc.smax);
  using L = SepLayout<cc.smax, cc.tile, P, st_depth>;
  auto kern = k_degrid_sep<smin, cc.smax, nt, cc.tile, P, st_depth>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, cc.nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "separable degridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, nt, L::bytes, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// Exact-support kernels (the kExactCand table): S is a compile-time constant and the row groups
// divide S, so every thread owns the same number of rows.
template <int S, int P, int C>
awg_status run_grid_exact(const GridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr ExactCfg e = exact_cfg(S, C);
  constexpr int nt = S * e.g_grid;
  static_assert(e.tile > 0 && S % e.g_grid == 0 && nt <= 1024 && e.stage >= 1 && e.stage <= nt,
                "bad exact-support configuration");
  using L = SepLayout<S, e.tile, P, e.stage>;
  static_assert(L::bytes <= 227 * 1024, "exact-support gridding window does not fit in shared memory");
  auto kern = k_grid_sep<S - 1, S, nt, e.tile, P, e.stage>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "exact-support gridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, nt, L::bytes, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

template <int S, int P, int C>
awg_status run_degrid_exact(const DegridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr ExactCfg e = exact_cfg(S, C);
  constexpr int nt = S * e.g_degrid;
  static_assert(e.tile > 0 && S % e.g_degrid == 0 && nt <= 1024 && e.stage >= 1 && e.stage <= nt,
                "bad exact-support configuration");
  using L = SepLayout<S, e.tile, P, e.stage>;
  static_assert(L::bytes <= 227 * 1024, "exact-support degridding window does not fit in shared memory");
  auto kern = k_degrid_sep<S - 1, S, nt, e.tile, P, e.stage>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "exact-support degridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, nt, L::bytes, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// Fused kernels for CF sets of RK = 2..4 outer-product terms on the exact supports (configuration
// 0): the staging depth is halved until the layout fits shared memory.
template <int S, int T, int P, int RK, int ST0>
constexpr int fused_stage() {
  if constexpr (SepLayout<S, T, P, ST0, RK>::bytes <= 227 * 1024 || ST0 <= 2) return ST0;
  else return fused_stage<S, T, P, RK, ST0 / 2>();
}

// Staging depth the fused kernels start from: configuration 0's, except where a sweep of the batched
// AW-projection workload (4 terms, 4 pols; per-launch times) found twice the depth faster:
// gridding at support 40 (45.4 -> 41.9 ms) and degridding at support 32 (31.9 -> 31.3 ms).  Deeper
// staging elsewhere cost occupancy (e.g. support 24: 18.4 -> 26 ms).
constexpr int fused_stage0(int S, int P, int RK, bool grid, int base) {
  return P == 4 && RK == 4 && ((grid && S == 40) || (!grid && S == 32)) ? 2 * base : base;
}

template <int S, int P, int RK, bool MIX = false, int C = 0>
awg_status run_grid_fused(const GridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr ExactCfg e = exact_cfg(S, C);
  constexpr int nt = S * e.g_grid;
  constexpr int stage = fused_stage<S, e.tile, P, RK, fused_stage0(S, P, RK, true, e.stage)>();
  using L = SepLayout<S, e.tile, P, stage, RK>;
  static_assert(L::bytes <= 227 * 1024, "fused gridding window does not fit in shared memory");
  auto kern = k_grid_sep<S - 1, S, nt, e.tile, P, stage, RK, MIX>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "fused gridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, nt, L::bytes, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

template <int S, int P, int RK, bool MIX = false, int C = 0>
awg_status run_degrid_fused(const DegridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr ExactCfg e = exact_cfg(S, C);
  constexpr int nt = S * e.g_degrid;
  constexpr int stage = fused_stage<S, e.tile, P, RK, fused_stage0(S, P, RK, false, e.stage)>();
  using L = SepLayout<S, e.tile, P, stage, RK>;
  static_assert(L::bytes <= 227 * 1024, "fused degridding window does not fit in shared memory");
  auto kern = k_degrid_sep<S - 1, S, nt, e.tile, P, stage, RK, MIX>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nt, L::bytes));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "fused degridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, nt, L::bytes, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

#define AWG_FOR_FUSED(M, RK)                                                                                \
  M(8, 1, RK) M(8, 2, RK) M(8, 4, RK) M(16, 1, RK) M(16, 2, RK) M(16, 4, RK) M(24, 1, RK) M(24, 2, RK)     \
  M(24, 4, RK) M(32, 1, RK) M(32, 2, RK) M(32, 4, RK) M(40, 1, RK) M(40, 2, RK) M(40, 4, RK) M(48, 1, RK) \
  M(48, 2, RK) M(48, 4, RK) M(56, 1, RK) M(56, 2, RK) M(56, 4, RK) M(64, 1, RK) M(64, 2, RK) M(64, 4, RK)
#define AWG_DECLARE_GRID_FUSED(S, P, RK) \
  extern template awg_status run_grid_fused<S, P, RK>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_FUSED(S, P, RK) \
  extern template awg_status run_degrid_fused<S, P, RK>(const DegridArgs&, int, int, cudaStream_t);
// configuration 1 (the tiles and staging of exact-support candidate 1) of the fused kernels
#define AWG_DECLARE_GRID_FUSED_C1(S, P, RK) \
  extern template awg_status run_grid_fused<S, P, RK, false, 1>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_FUSED_C1(S, P, RK) \
  extern template awg_status run_degrid_fused<S, P, RK, false, 1>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_FUSED_C1(S, P, RK) \
  template awg_status run_grid_fused<S, P, RK, false, 1>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_FUSED_C1(S, P, RK) \
  template awg_status run_degrid_fused<S, P, RK, false, 1>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_FUSED(S, P, RK) \
  template awg_status run_grid_fused<S, P, RK>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_FUSED(S, P, RK) \
  template awg_status run_degrid_fused<S, P, RK>(const DegridArgs&, int, int, cudaStream_t);
// The pol-mixing instances (full-polarisation base passes): 4 pols, every exact support.
#define AWG_FOR_FUSED_MIX(M, RK) M(8, 4, RK) M(16, 4, RK) M(24, 4, RK) M(32, 4, RK) M(40, 4, RK) M(48, 4, RK) M(56, 4, RK) M(64, 4, RK)
#define AWG_DECLARE_GRID_FUSED_MIX(S, P, RK) \
  extern template awg_status run_grid_fused<S, P, RK, true>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_FUSED_MIX(S, P, RK) \
  extern template awg_status run_degrid_fused<S, P, RK, true>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_FUSED_MIX(S, P, RK) \
  template awg_status run_grid_fused<S, P, RK, true>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_FUSED_MIX(S, P, RK) \
  template awg_status run_degrid_fused<S, P, RK, true>(const DegridArgs&, int, int, cudaStream_t);

#define AWG_FOR_EXACT_AND_POLS(M, C)                                                                        \
  M(8, 1, C) M(8, 2, C) M(8, 4, C) M(16, 1, C) M(16, 2, C) M(16, 4, C) M(24, 1, C) M(24, 2, C) M(24, 4, C)      \
  M(32, 1, C) M(32, 2, C) M(32, 4, C) M(40, 1, C) M(40, 2, C) M(40, 4, C) M(48, 1, C) M(48, 2, C) M(48, 4, C) \
  M(56, 1, C) M(56, 2, C) M(56, 4, C) M(64, 1, C) M(64, 2, C) M(64, 4, C)
#define AWG_DECLARE_GRID_EXACT(S, P, C) \
  extern template awg_status run_grid_exact<S, P, C>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_EXACT(S, P, C) \
  extern template awg_status run_degrid_exact<S, P, C>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_EXACT(S, P, C) \
  template awg_status run_grid_exact<S, P, C>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_EXACT(S, P, C) \
  template awg_status run_degrid_exact<S, P, C>(const DegridArgs&, int, int, cudaStream_t);

#define AWG_FOR_SEP_CLASSES_AND_POLS(M) \
  M(0, 1) M(0, 2) M(0, 4) M(1, 1) M(1, 2) M(1, 4) M(2, 1) M(2, 2) M(2, 4) M(3, 1) M(3, 2) M(3, 4) M(4, 1) M(4, 2) M(4, 4) \
  M(5, 1) M(5, 2) M(5, 4)

#define AWG_DECLARE_GRID_SEP(C, P) \
  extern template awg_status run_grid_sep<C, P>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_SEP(C, P) \
  extern template awg_status run_degrid_sep<C, P>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_SEP(C, P) template awg_status run_grid_sep<C, P>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_SEP(C, P) \
  template awg_status run_degrid_sep<C, P>(const DegridArgs&, int, int, cudaStream_t);

}  // namespace awg
