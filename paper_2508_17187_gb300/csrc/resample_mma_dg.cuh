// Degridding on the tensor cores (tcgen05, sm_103a) for separable rank-1 CF records on the exact
// supports with windows of side U <= 64: the degridding half of configuration 3.
//
// With separable CFs, sample j of a work item reads V_jp = conj(ph_j) sum_x fx_j[x - dx_j]
// T_j(x, p) with T_j(x, p) = sum_y fy_j[y - dy_j] G(X0 + x, Y0 + y, p) (the sum of Eq.
// ME-MOD-GRIDDED over the sample's S x S footprint, the CF being fx times fy).  T is a dense
// product over y for up to 64 samples at once.  In real arithmetic, with row m = (j, c) (c: real
// / imaginary part), column n = (x, p) and k = (y, c'):
//   A[(j,0)][(y,0)] = Re f, A[(j,0)][(y,1)] = -Im f, A[(j,1)][(y,0)] = Im f, A[(j,1)][(y,1)] = Re f,
//   (f = fy_j[y - dy_j], zero outside the footprint), B[(x,p)][(y,0)] = Re G, B[(x,p)][(y,1)] = Im G,
// D = A B^T holds Re T in rows c = 0 and Im T in rows c = 1 (M = 128 rows: 64 samples; N = U P).
// The window is never held whole: the producer loads it by TMA in slices of KY rows of y, and
// each slice is one K block of the product (the window of an item is read once per pass of 64 of
// its samples).  The sum over x runs in the epilogue, one lane per (sample, part), with fx read
// from the L2-resident factor table.
//
// Precision: 3xTF32 split products with FP32 accumulation, as in the tensor-core gridding.
//
// Roles (one persistent CTA per SM): warp 0 the producer (stages of 64 samples: first-tap
// offsets, output rows, phasors, fx row offsets and the fy rows; window slices by TMA), warp 1 the
// tensor memory and the MMA issuer, warps 2-5 the epilogue, the rest the builders of the A and B
// operands.  Every hand-off is an mbarrier phase with a bounded wait (ws_sync.cuh).
#pragma once

#include "resample_mma.cuh"

namespace awg {

// ST = 64 samples per pass; KY window rows per slice; D stages, NZ slice buffers, NOB operand
// buffers.
template <int S, int P, int TILE, int KY, int D, int NZ, int NOB>
struct MmaDgLayout {
  static constexpr int ST = 64;
  static constexpr int KY_ = KY, D_ = D, NZ_ = NZ, NOB_ = NOB;
  static constexpr int U = TILE + S - 1;
  static_assert(U <= 64 && U % KY == 0 && KY % 8 == 0, "slices of KY rows cover the window");
  static constexpr int N = U * P;                                   // MMA N: columns (x, p)
  static_assert(N % 16 == 0 && N <= 256, "MMA N of a 128-row tile: a multiple of 16, at most 256");
  static constexpr int NSL = U / KY;                                // slices per pass
  static constexpr int K = 2 * KY, KS = K / 8, KQ = KY / 2;
  static constexpr int NACC = 2;
  static constexpr int TCOLS = 2 * N <= 32 ? 32 : 2 * N <= 64 ? 64 : 2 * N <= 128 ? 128 : 2 * N <= 256 ? 256 : 512;
  static constexpr unsigned LBO = 128, SBO = (K / 4) * 128;
  // P = 1 window rows: UB pixels from the even pixel at or below X0 (see the warp-specialised
  // degridding layout: a 2-D TMA box must start at a 16-byte x coordinate)
  static constexpr int XA = (P == 1 && TILE % 2 == 1) ? 1 : 0;
  static constexpr int UB = (P == 1) ? ((U + XA + 1) & ~1) : U;
  static constexpr unsigned slice_box_bytes = (unsigned)KY * UB * P * 8;
  static constexpr size_t slice_bytes = ws_al1k(slice_box_bytes);
  static constexpr size_t a_bytes = (size_t)128 * K * 4;
  static constexpr size_t b_bytes = (size_t)N * K * 4;
  static constexpr size_t ob_ahi = 0, ob_alo = a_bytes, ob_bhi = 2 * a_bytes, ob_blo = 2 * a_bytes + b_bytes;
  static constexpr size_t ob_hdr = 2 * a_bytes + 2 * b_bytes;
  static constexpr size_t ob_bytes = ws_al1k(ob_hdr + 16);
  // stage: header, first-tap offsets, output rows, phasors, fx row offsets, fy rows
  static constexpr size_t st_pk = 16;
  static constexpr size_t st_src = st_pk + 4 * ST;
  static constexpr size_t st_ph = st_src + 4 * ST;
  static constexpr size_t st_fxo = st_ph + 8 * ST;
  static constexpr size_t st_fy = st_fxo + 8 * ST;
  static constexpr int RS = S + 2;   // fy rows RS values apart (bank spread, as for gridding)
  static constexpr size_t stage_bytes = ws_al16(st_fy + (size_t)ST * RS * 8);
  static constexpr int NB_WARPS = 14;
  static constexpr int NT = 32 * (2 + 4 + NB_WARPS);
  static constexpr size_t off_ob = 0;
  static constexpr size_t off_slice = NOB * ob_bytes;
  static constexpr size_t off_stage = off_slice + NZ * slice_bytes;
  static constexpr size_t off_bar = off_stage + D * stage_bytes;
  // barriers: full[D], empty[D], zfull[NZ], zempty[NZ], ofull[NOB], oempty[NOB], afull[2], aempty[2], fin
  static constexpr size_t off_misc = off_bar + 8 * (2 * D + 2 * NZ + 2 * NOB + 2 * NACC + 1);
  static constexpr size_t off_soff = ws_al16(off_misc + 32 + 4 * NACC);
  static constexpr size_t bytes = off_soff + 8 * (size_t)kSepOffCache;
  static constexpr size_t alloc = (bytes + 1024 > 116 * 1024 ? bytes + 1024 : 116 * 1024);
};

// The producer warp: per pass, a stage of up to 64 samples of one item (two per lane) and the
// item's window in NSL slices of KY rows (TMA tile loads into the slice ring).  A stage with
// nst = -1 ends the work.
template <int S, int P, int TILE, class L>
__device__ __forceinline__ void mma_dg_producer(const DegridArgs& a, const int cls, const CUtensorMap* gmap,
                                                unsigned char* smem, uint64_t* full, uint64_t* empty,
                                                uint64_t* zfull, uint64_t* zempty, const int64_t* offs,
                                                volatile int* abort_flag, unsigned long long* err, const int lane) {
  constexpr int ST = L::ST, D = L::D_, NZ = L::NZ_;
  constexpr bool kRowsByPieces = S <= 64;   // every exact support (one row per sample); bulk copies beyond
  WsItemWalker walk;
  walk.init(a.class_range[cls], a.class_range[cls + 1], cls, TILE, ST, a.queue, a.items);
  const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
  auto rec_at = [&](const WsChunk& d, int i) {
    SampleRec r{};
    if (d.valid && i < d.nst) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(a.rec + d.start + i));
      r = *reinterpret_cast<const SampleRec*>(&v);
    }
    return r;
  };
  auto ph_at = [&](const WsChunk& d, const SampleRec& rc, int i) {
    return (a.phasor && d.valid && i < d.nst) ? __ldg(a.phasor + rc.src) : make_float2(1.f, 0.f);
  };
  // records three passes ahead, phasors one
  WsChunk d0 = walk.next(), d1 = walk.next(), d2 = walk.next();
  SampleRec r0a = rec_at(d0, lane), r0b = rec_at(d0, lane + 32);
  SampleRec r1a = rec_at(d1, lane), r1b = rec_at(d1, lane + 32);
  SampleRec r2a = rec_at(d2, lane), r2b = rec_at(d2, lane + 32);
  float2 ph0a = ph_at(d0, r0a, lane), ph0b = ph_at(d0, r0b, lane + 32);
  int k = 0, zc = 0;
  int zuse[NZ];   // last use of each slice buffer (its zfull phase), -1: never loaded
#pragma unroll
  for (int z = 0; z < NZ; ++z) zuse[z] = -1;
  bool ok = true;
  while (d0.valid) {
    const int s = k % D;
    unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
    if (!warp_wait(empty + s, ((k / D) & 1) ^ 1, abort_flag, err)) {
      ok = false;
      break;
    }
    const int X0 = d0.xy & 0xffff, Y0 = d0.xy >> 16;
    long long fyo[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h;
      const SampleRec& r = h ? r0b : r0a;
      if (i < d0.nst) {
        reinterpret_cast<int*>(sg + L::st_pk)[i] = (r.p0x - X0) | ((r.p0y - Y0) << 8);
        reinterpret_cast<int*>(sg + L::st_src)[i] = a.rank > 1 ? r.src * a.rank + r.cf % a.rank : r.src;
        reinterpret_cast<float2*>(sg + L::st_ph)[i] = h ? ph0b : ph0a;
        long long fxo;
        ws_rows<S>(offs, a.cf_shift, a.OS, r, fxo, fyo[h]);
        reinterpret_cast<long long*>(sg + L::st_fxo)[i] = fxo;
        if constexpr (!kRowsByPieces) {
          fence_proxy_async_smem();
          bulk_load(sg + L::st_fy + (size_t)i * L::RS * 8, sep2 + fyo[h], S * 8, full + s);
        }
      }
    }
    if constexpr (kRowsByPieces) {
      // fy rows: each lane copies its two samples' rows in 16-byte pieces (measured faster than one
      // bulk copy per row for every support)
      constexpr int HP = S / 2;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < d0.nst) {
          unsigned char* dst = sg + L::st_fy + (size_t)i * L::RS * 8;
#pragma unroll
          for (int w = 0; w < HP; ++w) cp_async16(dst + 16 * w, sep2 + fyo[h] + 2 * w);
        }
      }
    }
    if (lane == 0) *reinterpret_cast<WsHeader*>(sg) = WsHeader{d0.nst, d0.flags, d0.xy, 0};
    if (!(a.withhold && k == 0)) {
      if (!kRowsByPieces && lane == 0) {
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(full + s)) : "memory");
        mbar_arrive_expect_tx(full + s, (unsigned)(d0.nst * S * 8));
      } else {
        stage_arrive(full + s);
      }
    }
    // the window of the pass, slice by slice
    for (int sl = 0; sl < L::NSL; ++sl, ++zc) {
      const int z = zc % NZ;
      if (!warp_wait(zempty + z, ((zc / NZ) & 1) ^ 1, abort_flag, err)) {
        ok = false;
        break;
      }
      if (lane == 0) {
        fence_proxy_async_smem();
        unsigned char* dst = smem + L::off_slice + (size_t)z * L::slice_bytes;
        mbar_arrive_expect_tx(zfull + z, L::slice_box_bytes);
        if constexpr (P == 1) tma_load_2d(dst, gmap, 2 * (X0 & ~1), Y0 + sl * L::KY_, zfull + z);
        else tma_load_3d(dst, gmap, 0, X0, Y0 + sl * L::KY_, zfull + z);
      }
      zuse[z] = zc / NZ;
    }
    if (!ok) break;
    const WsChunk d3 = walk.next();
    const SampleRec r3a = rec_at(d3, lane), r3b = rec_at(d3, lane + 32);
    ph0a = ph_at(d1, r1a, lane);
    ph0b = ph_at(d1, r1b, lane + 32);
    d0 = d1;
    d1 = d2;
    d2 = d3;
    r0a = r1a;
    r0b = r1b;
    r1a = r2a;
    r1b = r2b;
    r2a = r3a;
    r2b = r3b;
    ++k;
  }
  if (ok && warp_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
    if (lane == 0) *reinterpret_cast<WsHeader*>(smem + L::off_stage + (size_t)(k % D) * L::stage_bytes) =
        WsHeader{-1, 0, 0, 0};
    stage_arrive(full + k % D);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (!ok || *abort_flag) {
    // no builder may wait for an issued slice any more: wait for the loads here (bounded)
    volatile int never = 0;
#pragma unroll
    for (int z = 0; z < NZ; ++z)
      if (zuse[z] >= 0) mbar_wait(zfull + z, zuse[z] & 1, &never, err);
  }
}

template <int S, int P, int TILE, int KY, int D, int NZ, int NOB>
__global__ void __launch_bounds__(MmaDgLayout<S, P, TILE, KY, D, NZ, NOB>::NT, 1)
    k_degrid_mma(const DegridArgs a, const int cls, const __grid_constant__ CUtensorMap gmap) {
  using L = MmaDgLayout<S, P, TILE, KY, D, NZ, NOB>;
  constexpr int KS = L::KS, KQ = L::KQ, N = L::N, NACC = L::NACC, NSL = L::NSL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  int64_t* s_off = reinterpret_cast<int64_t*>(smem + L::off_soff);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* empty = full + D;
  uint64_t* zfull = empty + D;
  uint64_t* zempty = zfull + NZ;
  uint64_t* ofull = zempty + NZ;
  uint64_t* oempty = ofull + NOB;
  uint64_t* afull = oempty + NOB;
  uint64_t* aempty = afull + NACC;
  uint64_t* fin = aempty + NACC;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::off_misc);
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(smem + L::off_misc + 16);
  int* acc_tag = reinterpret_cast<int*>(smem + L::off_misc + 32);   // [NACC] 1: a pass, -1: the end
  unsigned long long* err = a.err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const bool off_cached = a.n_sep_off <= kSepOffCache;
  if (off_cached)
    for (int i = tid; i < a.n_sep_off; i += L::NT) s_off[i] = a.sep_off[i];
  const int64_t* offs = off_cached ? s_off : a.sep_off;
  if (tid == 0) {
    for (int d = 0; d < D; ++d) {
      mbar_init(full + d, 64);   // the producer lanes, then their copies
      mbar_init(empty + d, 4);   // the epilogue warps
    }
    for (int z = 0; z < NZ; ++z) {
      mbar_init(zfull + z, 1);
      mbar_init(zempty + z, L::NB_WARPS);
    }
    for (int b = 0; b < NOB; ++b) {
      mbar_init(ofull + b, L::NB_WARPS);
      mbar_init(oempty + b, 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(afull + b, 2);   // the MMA thread's arrival (tag written) + the commit
      mbar_init(aempty + b, 4);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 0 && lane == 0) prefetch_tensormap(&gmap);
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((unsigned)L::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------------------------ producer
    mma_dg_producer<S, P, TILE, L>(a, cls, &gmap, smem, full, empty, zfull, zempty, offs, abort_flag, err, lane);
  } else if (warp == 1) {
    // ------------------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr unsigned idesc = umma_idesc_tf32(128, N);
      int pass = 0;
      bool ok = true;
      for (int q = 0;; ++q) {
        const int ob = q % NOB;
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        if (!mbar_wait(ofull + ob, (q / NOB) & 1, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int4 hdr = *reinterpret_cast<const int4*>(obuf + L::ob_hdr);   // nst, slice
        if (hdr.x < 0) break;
        const int ab = pass % NACC;
        if (hdr.y == 0) {
          if (!mbar_wait(aempty + ab, ((pass / NACC) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const unsigned abase = smem_u32(obuf);
        const uint64_t dah = umma_sdesc(abase + (unsigned)L::ob_ahi, L::LBO, L::SBO);
        const uint64_t dal = umma_sdesc(abase + (unsigned)L::ob_alo, L::LBO, L::SBO);
        const uint64_t dbh = umma_sdesc(abase + (unsigned)L::ob_bhi, L::LBO, L::SBO);
        const uint64_t dbl = umma_sdesc(abase + (unsigned)L::ob_blo, L::LBO, L::SBO);
        const unsigned d = tmem + (unsigned)(ab * N);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const uint64_t o = (uint64_t)((ks * 2 * L::LBO) >> 4);
          umma_tf32(d, dal + o, dbh + o, idesc, (hdr.y == 0 && ks == 0) ? 0u : 1u);
          umma_tf32(d, dah + o, dbl + o, idesc, 1u);
          umma_tf32(d, dah + o, dbh + o, idesc, 1u);
        }
        umma_commit(oempty + ob);
        if (hdr.y == NSL - 1) {
          acc_tag[ab] = 1;
          mbar_arrive(afull + ab);
          umma_commit(afull + ab);
          ++pass;
        }
      }
      const int ab = pass % NACC;
      if (ok && mbar_wait(aempty + ab, ((pass / NACC) & 1) ^ 1, abort_flag, err)) {
        acc_tag[ab] = -1;
        mbar_arrive(afull + ab);
        mbar_arrive(afull + ab);
      }
      umma_commit(fin);
      volatile int never = 0;
      mbar_wait(fin, 0, &never, err);
    }
    __syncwarp();
  } else if (warp < 6) {
    // ------------------------------------------------------------------------------ epilogue
    // Lane m = 32 q + lane of the tensor memory holds part c = m mod 2 of T_j(x, p) for sample
    // j = m / 2 over the columns (x, p).  With w = fx_j[x - dx_j]: the real-part lane adds
    // (Re w) Re T to Re V and (Im w) Re T to Im V, the imaginary-part lane -(Im w) Im T and
    // (Re w) Im T; one exchange between the two lanes completes V_jp.
    const int q = warp & 3;
    const int jl = 16 * q + (lane >> 1), c = lane & 1;
    const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
    for (int k = 0;; ++k) {
      const int ab = k % NACC;
      if (!warp_wait(afull + ab, (k / NACC) & 1, abort_flag, err)) break;
      tc_fence_after();
      if (acc_tag[ab] < 0) break;
      const int s = k % D;
      const unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      const bool valid = jl < h.nst;
      int dx = 0;
      const float2* fxr = sep2;
      if (valid) {
        dx = reinterpret_cast<const int*>(sg + L::st_pk)[jl] & 0xff;
        fxr = sep2 + reinterpret_cast<const long long*>(sg + L::st_fxo)[jl];
      }
      float vr[P], vi[P];
#pragma unroll
      for (int p = 0; p < P; ++p) vr[p] = vi[p] = 0.f;
      for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(ab * N + n0), v);
        if (valid) {
#pragma unroll
          for (int g = 0; g < 16 / P; ++g) {
            const int tx = n0 / P + g - dx;
            if (tx >= 0 && tx < S) {
              const float2 w = __ldg(fxr + tx);
              const float wa = c ? -w.y : w.x, wb = c ? w.x : w.y;
#pragma unroll
              for (int p = 0; p < P; ++p) {
                vr[p] = fmaf(wa, v[g * P + p], vr[p]);
                vi[p] = fmaf(wb, v[g * P + p], vi[p]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        vr[p] += __shfl_xor_sync(0xffffffffu, vr[p], 1);
        vi[p] += __shfl_xor_sync(0xffffffffu, vi[p], 1);
      }
      if (valid && c == 0) {
        const float2 ph = reinterpret_cast<const float2*>(sg + L::st_ph)[jl];
        const int src = reinterpret_cast<const int*>(sg + L::st_src)[jl];
        float* o = a.vis_out + ((size_t)src * a.vstride + a.voff) * 2;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float orr = vr[p] * ph.x + vi[p] * ph.y, oi = vi[p] * ph.x - vr[p] * ph.y;   // V conj(ph)
          if (a.accumulate > 0) {
            o[2 * p] += orr;
            o[2 * p + 1] += oi;
          } else if (a.accumulate < 0) {   // residual: V - D(grid)
            o[2 * p] -= orr;
            o[2 * p + 1] -= oi;
          } else {
            o[2 * p] = orr;
            o[2 * p + 1] = oi;
          }
        }
      }
      tc_fence_before();
      warp_arrive(aempty + ab);
      warp_arrive(empty + s);
    }
  } else {
    // ------------------------------------------------------------------------------ builders
    // A task (row m = (j, c), K group kq) holds rows y = KY sl + 2 kq, + 1 of sample j's fy:
    // (Re f, -Im f) in row c = 0 and (Im f, Re f) in row c = 1.  A B task (row n = (x, p)) holds
    // (Re G, Im G) of the slice at those rows.  Eight consecutive rows per K group, so that the
    // 16-byte stores of a warp fall in all eight bank groups.
    const int bt = tid - 6 * 32;
    constexpr int NBT = 32 * L::NB_WARPS;
    int q = 0, zc = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int s = k % D;
      const unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
      if (!warp_wait(full + s, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      if (h.nst < 0) {
        const int ob = q % NOB;
        if (!warp_wait(oempty + ob, ((q / NOB) & 1) ^ 1, abort_flag, err)) break;
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        if (bt == 0) *reinterpret_cast<int4*>(obuf + L::ob_hdr) = make_int4(-1, 0, 0, 0);
        warp_arrive(ofull + ob);
        break;
      }
      const int* pkv = reinterpret_cast<const int*>(sg + L::st_pk);
      const float2* fyv = reinterpret_cast<const float2*>(sg + L::st_fy);
      const int xa = (P == 1) ? ((h.xy & 0xffff) & L::XA) : 0;   // window column 0 in a P = 1 slice row
      for (int sl = 0; sl < NSL; ++sl, ++q, ++zc) {
        const int z = zc % NZ, ob = q % NOB;
        if (!warp_wait(zfull + z, (zc / NZ) & 1, abort_flag, err) ||
            !warp_wait(oempty + ob, ((q / NOB) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        const float2* slice = reinterpret_cast<const float2*>(smem + L::off_slice + (size_t)z * L::slice_bytes);
        if (bt == 0) *reinterpret_cast<int4*>(obuf + L::ob_hdr) = make_int4(h.nst, sl, 0, 0);
#pragma unroll 4
        for (int task = bt; task < 128 * KQ; task += NBT) {
          const int kq = (task >> 3) % KQ;
          const int m = (task / (8 * KQ)) * 8 + (task & 7);
          const int j = m >> 1, c = m & 1;
          float e[4];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            float fr = 0.f, fi = 0.f;
            if (j < h.nst) {
              const int ty = KY * sl + 2 * kq + h2 - ((pkv[j] >> 8) & 0xff);
              if (ty >= 0 && ty < S) {
                const float2 f = fyv[j * L::RS + ty];
                fr = f.x;
                fi = f.y;
              }
            }
            e[2 * h2] = c ? fi : fr;
            e[2 * h2 + 1] = c ? fr : -fi;
          }
          float hi[4], lo[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) tf32_split(e[i], hi[i], lo[i]);
          const size_t off = (size_t)(m % 8) * 16 + (size_t)(m / 8) * L::SBO + (size_t)kq * L::LBO;
          *reinterpret_cast<float4*>(obuf + L::ob_ahi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4*>(obuf + L::ob_alo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
#pragma unroll 4
        for (int task = b_first<128 * KQ, NBT>(bt); task < N * KQ; task += NBT) {
          const int kq = (task >> 3) % KQ;
          const int nn = (task / (8 * KQ)) * 8 + (task & 7);
          const int x = nn / P, p = nn % P;
          float e[4];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int yy = 2 * kq + h2;
            const float2 g = (P == 1) ? slice[yy * L::UB + x + xa] : slice[(yy * L::U + x) * P + p];
            e[2 * h2] = g.x;
            e[2 * h2 + 1] = g.y;
          }
          float hi[4], lo[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) tf32_split(e[i], hi[i], lo[i]);
          const size_t off = (size_t)(nn % 8) * 16 + (size_t)(nn / 8) * L::SBO + (size_t)kq * L::LBO;
          *reinterpret_cast<float4*>(obuf + L::ob_bhi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4*>(obuf + L::ob_blo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_proxy_async_smem();
        warp_arrive(ofull + ob);
        warp_arrive(zempty + z);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  __syncwarp();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)L::TCOLS));
}

// Tensor-core degridding configuration per exact support and pol count (windows up to 64): the
// tile (as for gridding), window rows per slice, stages, slice buffers, operand buffers.
struct MmaDgCfg {
  int S, P, tile, ky, d, nz, nob;
};
constexpr MmaDgCfg kMmaDgCfg[21] = {
    {8, 1, 9, 16, 4, 3, 3},   {8, 2, 9, 16, 4, 3, 3},   {8, 4, 9, 16, 4, 3, 3},   {16, 1, 17, 16, 4, 3, 3},
    {16, 2, 17, 16, 4, 3, 3}, {16, 4, 17, 16, 4, 3, 2}, {24, 1, 9, 16, 4, 3, 3},  {24, 2, 9, 16, 3, 3, 3},
    {24, 4, 9, 16, 3, 3, 2},  {32, 1, 17, 16, 3, 3, 3}, {32, 2, 17, 16, 4, 2, 2}, {32, 4, 17, 8, 3, 3, 3},
    {40, 1, 9, 16, 3, 3, 3},  {40, 2, 9, 16, 3, 3, 2},  {40, 4, 9, 8, 2, 3, 3},   {48, 1, 17, 16, 2, 2, 3},
    {48, 2, 17, 16, 2, 2, 2}, {48, 4, 17, 8, 2, 3, 2},  {56, 1, 9, 16, 3, 3, 2},  {56, 2, 9, 16, 2, 2, 2},
    {56, 4, 9, 8, 2, 3, 2},
};
constexpr MmaDgCfg mma_dg_cfg(int S, int P) {
  for (const MmaDgCfg& e : kMmaDgCfg)
    if (e.S == S && e.P == P) return e;
  return MmaDgCfg{S, P, 0, 0, 0, 0, 0};
}

template <int S, int P>
awg_status run_degrid_mma(const DegridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr MmaDgCfg c = mma_dg_cfg(S, P);
  static_assert(c.tile == exact_cfg(S, 3).tile, "the plan bins candidate 3 by this tile");
  using L = MmaDgLayout<S, P, c.tile, c.ky, c.d, c.nz, c.nob>;
  static_assert(L::alloc <= 227 * 1024, "tensor-core degridding stages do not fit");
  auto kern = k_degrid_mma<S, P, c.tile, c.ky, c.d, c.nz, c.nob>;
  static int ready = 0;
  if (!ready) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::alloc));
    int bps = 0;
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, L::NT, L::alloc));
    if (bps != 1) return set_error(AWG_ERR_CUDA, "tensor-core degridding kernel must hold an SM alone");
    ready = 1;
  }
  CUtensorMap map;
  awg_status s = make_grid_tensor_map(&map, a.grid, a.N, P, L::U, L::UB, c.ky);
  if (s != AWG_OK) return s;
  kern<<<sms, L::NT, L::alloc, st>>>(a, slot, map);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

#define AWG_FOR_MMA_DG_A(M) M(8, 1) M(8, 2) M(8, 4) M(16, 1) M(16, 2) M(16, 4) M(24, 1) M(24, 2) M(24, 4) \
  M(32, 1) M(32, 2) M(32, 4)
#define AWG_FOR_MMA_DG_B(M) M(40, 1) M(40, 2) M(40, 4) M(48, 1) M(48, 2) M(48, 4) M(56, 1) M(56, 2) M(56, 4)
#define AWG_DECLARE_DEGRID_MMA(S, P) extern template awg_status run_degrid_mma<S, P>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_MMA(S, P) template awg_status run_degrid_mma<S, P>(const DegridArgs&, int, int, cudaStream_t);

}  // namespace awg
