// Gridding on the tensor cores (tcgen05, sm_103a) for separable rank-1 CF records on the exact
// supports: configuration 3 of cf_set_autotune / cf_set_choose.
//
// With separable CFs the gridding of one work item is a dense product.  Sample j of the item adds
// Y_j(y) X_j(x, p) to window pixel (x, y) of pol p, with Y_j(y) = conj(fy_j[y - dy_j]) and
// X_j(x, p) = conj(fx_j[x - dx_j]) w_jp V_jp (zero outside the sample's S x S footprint), so the
// window is W = sum_j X_j Y_j^T, a GEMM over the samples.  In real arithmetic, with row
// m = (x, p, c) (c: real / imaginary part), column n = y and k = (j, c'):
//   A[(x,p,0)][(j,0)] = Re X, A[(x,p,0)][(j,1)] = Im X, A[(x,p,1)][(j,0)] = Im X, A[(x,p,1)][(j,1)] = -Re X,
//   B[y][(j,0)] = Re fy, B[y][(j,1)] = Im fy (= -Im Y),
// D = A B^T holds Re W in rows c = 0 and Im W in rows c = 1.  The window is padded to UX x UN
// pixels (UX: a multiple of 128 / 2P so that the rows fill 128-row MMA tiles; UN: a multiple of
// 16); the padding is zero work that the tensor cores do anyway.
//
// Precision: the operands are FP32 values split into a TF32 head (rounded to nearest) and the FP32
// remainder, which the tensor cores truncate to TF32; each k-step runs A_lo B_hi + A_hi B_lo +
// A_hi B_hi (the 3xTF32 scheme), which keeps the relative error of a product near 2^-21 (the
// dropped A_lo B_lo term and the remainders' truncation).  The sum over an item's samples runs in
// the FP32 accumulator of the tensor memory, one accumulation per MMA (3 K/8 per chunk): over an
// item of 1024 samples that is about 770 additions, whose rounding puts the relative RMS error of
// a window near sqrt(770) 2^-23, a few 1e-6, whatever the flush mode.
//
// Roles (one persistent CTA per SM):
//  * warp 0, the producer, stages up to 32 samples at a time (records, factor rows by cp.async or
//    bulk copies, w V times the phasor) into a ring of stages;
//  * the builder warps cut a stage into chunks of J samples and turn each chunk into the A and B
//    operands (hi and lo parts) in the canonical no-swizzle K-major layout of the tensor cores, in
//    a ring of operand buffers;
//  * warp 1 owns the tensor memory; its lane 0 issues the MMAs of each chunk into the item's
//    accumulator (two accumulators, so that one item's flush overlaps the next item's MMAs) and
//    commits them to the barriers that free the operand buffer and, at the end of an item, hand
//    the accumulator to the epilogue;
//  * four epilogue warps (one per tensor-memory lane quarter) read the accumulator and add it to the
//    grid (the flush modes of grid_visibilities: plain, compensated, FP64).
// Every hand-off is an mbarrier phase with a bounded wait (ws_sync.cuh); tensor memory is released
// on every path before the CTA exits.
#pragma once

#include "resample_ws.cuh"

namespace awg {

// ------------------------------------------------------------------------- tcgen05 primitives

// Shared-memory matrix descriptor of a K-major operand without swizzling: core matrices of 8 rows
// x 16 bytes; lbo = byte distance between core matrices adjacent in K, sbo = between adjacent
// groups of 8 rows.
__device__ __forceinline__ uint64_t umma_sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture family
  return d;                 // base offset 0, absolute LBO, layout 0: no swizzle
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands K-major.
__host__ __device__ constexpr unsigned umma_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(unsigned d_tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Arrive on `bar` once the tensor-core operations this thread issued so far have completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes (lane quarter warp % 4).  The
// load is a warp-collective (.sync.aligned) instruction: the warp is reconverged first.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 head of x and the FP32 remainder x - head.  TF32 keeps the sign, the 8 exponent bits and the
// top 10 mantissa bits of an FP32 value: adding half a unit of the 11th mantissa bit to the bit
// pattern and clearing the low 13 bits rounds the magnitude to nearest, ties away from zero
// (a carry into the exponent is the correct result), on the integer pipe rather than through a
// conversion.  The tensor cores read the remainder's top 19 bits (truncation: below 2^-21 of x).
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
  lo = x - hi;
}

// ------------------------------------------------------------------------------------- layout

// J samples per MMA chunk (K = 2 J), ST samples per producer stage (a stage is cut into ST / J
// chunks), D stages, NOB operand buffers.
template <int S, int P, int TILE, int J, int ST, int D, int NOB>
struct MmaGridLayout {
  static_assert(S % 2 == 0, "factor rows move in 16-byte units");
  static_assert(J % 8 == 0 && ST % J == 0 && ST <= 32, "chunks of whole K steps; a stage is one warp's samples");
  static constexpr int U = TILE + S - 1;                              // window side
  static constexpr int XQ = 128 / (2 * P);                            // pixels per 128-row tile
  static constexpr int UX = (U + XQ - 1) / XQ * XQ;                   // padded columns (x)
  static constexpr int UN = (U + 15) / 16 * 16;                       // padded rows (y): MMA N
  static constexpr int M = UX * P * 2;                                // A rows
  static constexpr int MT = M / 128;                                  // 128-row tiles
  static constexpr int K = 2 * J;                                     // per chunk
  static constexpr int KS = K / 8;                                    // MMA k-steps per chunk
  static constexpr int KQ = J / 2;                                    // 16-byte K groups per row
  static constexpr int NACC = (2 * MT * UN <= 512) ? 2 : 1;           // accumulators in tensor memory
  static constexpr int TCOLS0 = NACC * MT * UN;
  static constexpr int TCOLS = TCOLS0 <= 32 ? 32 : TCOLS0 <= 64 ? 64 : TCOLS0 <= 128 ? 128 : TCOLS0 <= 256 ? 256 : 512;
  static_assert(TCOLS0 <= 512, "the accumulator does not fit in tensor memory");
  static_assert(UN <= 256, "MMA N is at most 256");
  static_assert((UX * P) % 8 == 0, "A rows are built in groups of 8 pixel-pols");
  // canonical K-major layout: LBO = 128 bytes (adjacent core matrices in K), SBO = (K / 4) * 128
  static constexpr unsigned LBO = 128, SBO = (K / 4) * 128;
  static constexpr size_t a_bytes = (size_t)M * K * 4;
  static constexpr size_t b_bytes = (size_t)UN * K * 4;
  // operand buffer: A_hi, A_lo, B_hi, B_lo, then a small header (samples, flags, window origin)
  static constexpr size_t ob_ahi = 0, ob_alo = a_bytes, ob_bhi = 2 * a_bytes, ob_blo = 2 * a_bytes + b_bytes;
  static constexpr size_t ob_hdr = 2 * a_bytes + 2 * b_bytes;
  static constexpr size_t ob_bytes = ws_al1k(ob_hdr + 16);
  // producer stage: header, first-tap offsets, fy rows, fx rows, w V (times the phasor) per pol
  static constexpr size_t st_pk = 16;
  // staged factor rows RS = S + 2 values apart: the rows of consecutive samples start 8 banks apart,
  // so that the builders' reads of several samples' rows do not collide (rows stay 16-byte aligned)
  static constexpr int RS = S + 2;
  static constexpr size_t st_fy = st_pk + ws_al16(4 * ST);
  static constexpr size_t st_fx = st_fy + (size_t)ST * RS * 8;
  static constexpr size_t st_wv = st_fx + (size_t)ST * RS * 8;
  static constexpr size_t stage_bytes = ws_al16(st_wv + (size_t)ST * P * 8);
  static constexpr int NB_WARPS = 10;                                 // builders
  static constexpr int NT = 32 * (2 + 4 + NB_WARPS);                  // producer, MMA, epilogue, builders
  static constexpr size_t off_ob = 0;
  static constexpr size_t off_stage = NOB * ob_bytes;
  static constexpr size_t off_bar = off_stage + D * stage_bytes;
  // barriers: full[D], empty[D], ofull[NOB], oempty[NOB], afull[NACC], aempty[NACC], fin
  static constexpr size_t off_misc = off_bar + 8 * (2 * D + 2 * NOB + 2 * NACC + 1);
  static constexpr size_t off_soff = ws_al16(off_misc + 32 + 4 * NACC);
  static constexpr size_t bytes = off_soff + 8 * (size_t)kSepOffCache;
  // at least 116 KB so that one CTA holds an SM (and its tensor memory) alone
  static constexpr size_t alloc = (bytes + 1024 > 116 * 1024 ? bytes + 1024 : 116 * 1024);
};

// Warp-elected arrival: the warp's lanes have finished their part (their earlier shared-memory
// writes are ordered before lane 0's release by the warp barrier).
__device__ __forceinline__ void warp_arrive(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// Warp-uniform bounded wait: every lane waits, and the warp goes on only if all of its lanes saw
// the phase, so that a lane that gave up never leaves part of a warp at a warp-collective
// instruction (tcgen05.ld, shuffles, warp barriers) after the wait.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                          unsigned long long* err) {
  const bool ok = mbar_wait(bar, parity, abort_flag, err);
  return __all_sync(0xffffffffu, ok);
}

// Layout of the pols-in-N variant (windows of side U <= 64): A rows m = (x, c), x < 64 (M = 128,
// one MMA row tile), B rows (the MMA's N) n = (y, p) with p fastest, N = UY P, UY = U rounded up so
// that N is a multiple of 16.  The A operand then holds the conjugated x factor alone and B the
// conjugated y factor times w V, and every K step is one MMA per split term whatever P is.
template <int S, int P, int TILE, int J, int ST, int D, int NOB>
struct MmaNLayout {
  static_assert(S % 2 == 0, "factor rows move in 16-byte units");
  static_assert(J % 8 == 0 && ST % J == 0 && ST <= 32, "chunks of whole K steps; a stage is one warp's samples");
  static constexpr int U = TILE + S - 1;                              // window side
  static_assert(U <= 64, "the window's columns must fit one 128-row tile");
  static constexpr int YQ = 16 / P;                                   // rows per 16 columns of N
  static constexpr int UY = (U + YQ - 1) / YQ * YQ;
  static constexpr int N = UY * P;                                    // MMA N
  static_assert(N % 16 == 0 && N <= 256, "MMA N of a 128-row tile: a multiple of 16, at most 256");
  static constexpr int K = 2 * J, KS = K / 8, KQ = J / 2;
  static constexpr int NACC = 2;
  static constexpr int TCOLS = 2 * N <= 32 ? 32 : 2 * N <= 64 ? 64 : 2 * N <= 128 ? 128 : 2 * N <= 256 ? 256 : 512;
  static constexpr unsigned LBO = 128, SBO = (K / 4) * 128;
  static constexpr size_t a_bytes = (size_t)128 * K * 4;
  static constexpr size_t b_bytes = (size_t)N * K * 4;
  static constexpr size_t ob_ahi = 0, ob_alo = a_bytes, ob_bhi = 2 * a_bytes, ob_blo = 2 * a_bytes + b_bytes;
  static constexpr size_t ob_hdr = 2 * a_bytes + 2 * b_bytes;
  static constexpr size_t ob_bytes = ws_al1k(ob_hdr + 16);
  static constexpr size_t st_pk = 16;
  // staged factor rows RS = S + 2 values apart: the rows of consecutive samples start 8 banks apart,
  // so that the builders' reads of several samples' rows do not collide (rows stay 16-byte aligned)
  static constexpr int RS = S + 2;
  static constexpr size_t st_fy = st_pk + ws_al16(4 * ST);
  static constexpr size_t st_fx = st_fy + (size_t)ST * RS * 8;
  static constexpr size_t st_wv = st_fx + (size_t)ST * RS * 8;
  static constexpr size_t stage_bytes = ws_al16(st_wv + (size_t)ST * P * 8);
  static constexpr int NB_WARPS = 14;
  static constexpr int NT = 32 * (2 + 4 + NB_WARPS);
  static constexpr size_t off_ob = 0;
  static constexpr size_t off_stage = NOB * ob_bytes;
  static constexpr size_t off_bar = off_stage + D * stage_bytes;
  static constexpr size_t off_misc = off_bar + 8 * (2 * D + 2 * NOB + 2 * NACC + 1);
  static constexpr size_t off_soff = ws_al16(off_misc + 32 + 4 * NACC);
  static constexpr size_t bytes = off_soff + 8 * (size_t)kSepOffCache;
  static constexpr size_t alloc = (bytes + 1024 > 116 * 1024 ? bytes + 1024 : 116 * 1024);
};

// The builders' A and B tasks of one chunk form one list, A tasks first, dealt to the NBT builder
// threads in turn: thread t takes list entries t, t + NBT, ...  Its first B task is then the first
// such entry at or past the TA A tasks, less TA, so the threads left with one A task fewer take the
// next B tasks and no thread holds two more tasks than another.  TA and NBT are multiples of 32,
// so every warp still takes 32 consecutive tasks of each kind.
template <int TA, int NBT>
__device__ __forceinline__ int b_first(int t) {
  static_assert(TA % 32 == 0 && NBT % 32 == 0, "whole warps of tasks");
  constexpr int R = TA % NBT;
  return t >= R ? t - R : t + NBT - R;
}

// Adds one complex value pair to the grid: 16 bytes at `g` (pols p, p + 1 of a pixel, P >= 2) in the
// flush mode of grid_visibilities (0 plain, 1 compensated with the error into glo, 2 FP64 grid).
__device__ __forceinline__ void mma_flush4(float* grid, float* grid_lo, size_t e, int mode, float4 v) {
  if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) return;
  if (mode == 0) {
    atomicAdd(reinterpret_cast<float4*>(grid + e), v);
  } else if (mode == 1) {
    const float4 old = atomicAdd(reinterpret_cast<float4*>(grid + e), v);
    float er[4];
    const float o[4] = {old.x, old.y, old.z, old.w}, a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float sum = o[i] + a[i], bb = sum - o[i];
      er[i] = (o[i] - (sum - bb)) + (a[i] - bb);
    }
    if (er[0] != 0.f || er[1] != 0.f || er[2] != 0.f || er[3] != 0.f)
      atomicAdd(reinterpret_cast<float4*>(grid_lo + e), make_float4(er[0], er[1], er[2], er[3]));
  } else {
    double* g = reinterpret_cast<double*>(grid) + e;
    atomicAdd(g, (double)v.x);
    atomicAdd(g + 1, (double)v.y);
    atomicAdd(g + 2, (double)v.z);
    atomicAdd(g + 3, (double)v.w);
  }
}

// One complex value (8 bytes at `g`), as mma_flush4.
__device__ __forceinline__ void mma_flush2(float* grid, float* grid_lo, size_t e, int mode, float2 v) {
  if (v.x == 0.f && v.y == 0.f) return;
  if (mode == 0) {
    atomicAdd(reinterpret_cast<float2*>(grid + e), v);
  } else if (mode == 1) {
    const float2 old = atomicAdd(reinterpret_cast<float2*>(grid + e), v);
    const float sx = old.x + v.x, bx = sx - old.x, sy = old.y + v.y, by = sy - old.y;
    const float2 er = make_float2((old.x - (sx - bx)) + (v.x - bx), (old.y - (sy - by)) + (v.y - by));
    if (er.x != 0.f || er.y != 0.f) atomicAdd(reinterpret_cast<float2*>(grid_lo + e), er);
  } else {
    double* g = reinterpret_cast<double*>(grid) + e;
    atomicAdd(g, (double)v.x);
    atomicAdd(g + 1, (double)v.y);
  }
}


// 16-byte asynchronous copy global -> shared (L2 only), completion tracked per thread.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// A producer lane's two arrivals on a stage's full barrier (count 64 for the warp): one now
// (release of its plain shared-memory stores) and one when its cp.async copies have landed (at
// once when it has none).  Bulk copies add their bytes to the transaction count instead.
__device__ __forceinline__ void stage_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
  mbar_arrive(bar);
}

// The producer warp of the tensor-core gridding kernels: walks the CTA's items in stages of up to
// ST samples (one per lane): first-tap offsets in the window, the fx and fy factor rows (16-byte
// cp.async pieces for short rows, one bulk copy per row for long ones, completing on the stage's
// full barrier), w V times the phasor per pol; a stage with
// nst = -1 ends the work.  Adds the CTA's share of the sum of weights.
template <int S, int P, int TILE, int ST, int D, class L>
__device__ __forceinline__ void mma_producer(const GridArgs& a, const int cls, unsigned char* smem, uint64_t* full,
                                             uint64_t* empty, const int64_t* offs, volatile int* abort_flag,
                                             unsigned long long* err, const int lane) {
  constexpr bool kRowsByPieces = S <= 40;   // else one bulk copy per factor row (measured faster there)
  double wsum[P];
#pragma unroll
  for (int p = 0; p < P; ++p) wsum[p] = 0.0;
  WsItemWalker walk;
  walk.init(a.class_range[cls], a.class_range[cls + 1], cls, TILE, ST, a.queue, a.items);
  const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
  WsChunk d0 = walk.next();
  WsChunk d1 = walk.next();
  WsChunk d2 = walk.next();
  SampleRec r0 = ws_load_rec(a.rec, d0, lane);
  SampleRec r1 = ws_load_rec(a.rec, d1, lane);
  SampleRec r2 = ws_load_rec(a.rec, d2, lane);
  WsVis<P> x0 = ws_load_vis<P>(a, d0, r0, lane);
  WsVis<P> x1 = ws_load_vis<P>(a, d1, r1, lane);
  int k = 0;
  bool ok = true;
  while (d0.valid) {
    const int s = k % D;
    unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
    if (!warp_wait(empty + s, ((k / D) & 1) ^ 1, abort_flag, err)) {
      ok = false;
      break;
    }
    long long fxo = 0, fyo = 0;
    if (lane < d0.nst) {
      const int X0 = d0.xy & 0xffff, Y0 = d0.xy >> 16;
      reinterpret_cast<int*>(sg + L::st_pk)[lane] = (r0.p0x - X0) | ((r0.p0y - Y0) << 8);
      ws_rows<S>(offs, a.cf_shift, a.OS, r0, fxo, fyo);
      if constexpr (!kRowsByPieces) {
        fence_proxy_async_smem();
        bulk_load(sg + L::st_fx + (size_t)lane * L::RS * 8, sep2 + fxo, S * 8, full + s);
        bulk_load(sg + L::st_fy + (size_t)lane * L::RS * 8, sep2 + fyo, S * 8, full + s);
      }
      float2* dst = reinterpret_cast<float2*>(sg + L::st_wv) + lane * P;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float xr = x0.w[p] * x0.v[p].x, xi = x0.w[p] * x0.v[p].y;
        dst[p] = make_float2(xr * x0.ph.x - xi * x0.ph.y, xr * x0.ph.y + xi * x0.ph.x);
      }
      if (a.rank == 1 || r0.cf % a.rank == 0) {
#pragma unroll
        for (int p = 0; p < P; ++p) wsum[p] += (double)x0.w[p];
      }
    }
    // factor rows of up to 320 bytes: each lane copies its sample's two rows in 16-byte
    // cp.async pieces (one bulk copy per row leaves this one warp issue-bound on the copies)
    if constexpr (kRowsByPieces) {
      constexpr int HP = S / 2;   // 16-byte pieces per row
      if (lane < d0.nst) {
        unsigned char* dx_ = sg + L::st_fx + (size_t)lane * L::RS * 8;
        unsigned char* dy_ = sg + L::st_fy + (size_t)lane * L::RS * 8;
#pragma unroll
        for (int w = 0; w < HP; ++w) {
          cp_async16(dx_ + 16 * w, sep2 + fxo + 2 * w);
          cp_async16(dy_ + 16 * w, sep2 + fyo + 2 * w);
        }
      }
    }
    if (lane == 0) *reinterpret_cast<WsHeader*>(sg) = WsHeader{d0.nst, d0.flags, d0.xy, 0};
    if (!(a.withhold && k == 0)) {
      if (!kRowsByPieces && lane == 0) {
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(full + s)) : "memory");
        mbar_arrive_expect_tx(full + s, (unsigned)(d0.nst * 2 * S * 8));
      } else {
        stage_arrive(full + s);
      }
    }
    const WsChunk d3 = walk.next();
    const SampleRec r3 = ws_load_rec(a.rec, d3, lane);
    const WsVis<P> x2 = ws_load_vis<P>(a, d2, r2, lane);
    d0 = d1;
    d1 = d2;
    d2 = d3;
    r0 = r1;
    r1 = r2;
    r2 = r3;
    x0 = x1;
    x1 = x2;
    ++k;
  }
  if (ok && warp_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
    if (lane == 0) *reinterpret_cast<WsHeader*>(smem + L::off_stage + (size_t)(k % D) * L::stage_bytes) =
        WsHeader{-1, 0, 0, 0};
    stage_arrive(full + k % D);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");   // no copy of this warp outlives the CTA
#pragma unroll
  for (int p = 0; p < P; ++p) {
    double v = wsum[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v != 0.0 && a.sumwt) atomicAdd(a.sumwt + p, v);
  }
}

template <int S, int P, int TILE, int J, int ST, int D, int NOB>
__global__ void __launch_bounds__(MmaGridLayout<S, P, TILE, J, ST, D, NOB>::NT, 1)
    k_grid_mma(const GridArgs a, const int cls) {
  using L = MmaGridLayout<S, P, TILE, J, ST, D, NOB>;
  constexpr int MT = L::MT, KS = L::KS, KQ = L::KQ, UN = L::UN, NACC = L::NACC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  int64_t* s_off = reinterpret_cast<int64_t*>(smem + L::off_soff);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* empty = full + D;
  uint64_t* ofull = full + 2 * D;
  uint64_t* oempty = ofull + NOB;
  uint64_t* afull = oempty + NOB;
  uint64_t* aempty = afull + NACC;
  uint64_t* fin = aempty + NACC;   // completion of every MMA issued, before the tensor memory is freed
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::off_misc);
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(smem + L::off_misc + 16);
  int* acc_xy = reinterpret_cast<int*>(smem + L::off_misc + 32);   // [NACC] window origin of each accumulator
  unsigned long long* err = a.err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const bool off_cached = a.n_sep_off <= kSepOffCache;
  if (off_cached)
    for (int i = tid; i < a.n_sep_off; i += L::NT) s_off[i] = a.sep_off[i];
  const int64_t* offs = off_cached ? s_off : a.sep_off;
  if (tid == 0) {
    for (int d = 0; d < D; ++d) {
      mbar_init(full + d, 64);   // the producer lanes, then their copies
      mbar_init(empty + d, L::NB_WARPS);
    }
    for (int b = 0; b < NOB; ++b) {
      mbar_init(ofull + b, L::NB_WARPS);
      mbar_init(oempty + b, 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(afull + b, 2);   // the MMA thread's arrival (window origin written) + the commit
      mbar_init(aempty + b, 4);  // the four epilogue warps
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
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
    mma_producer<S, P, TILE, ST, D, L>(a, cls, smem, full, empty, offs, abort_flag, err, lane);
  } else if (warp == 1) {
    // ------------------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr unsigned idesc = umma_idesc_tf32(128, UN);
      int item = 0;
      bool ok = true;
      for (int q = 0;; ++q) {
        const int ob = q % NOB;
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        if (!mbar_wait(ofull + ob, (q / NOB) & 1, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int4 hdr = *reinterpret_cast<const int4*>(obuf + L::ob_hdr);   // nst, flags, xy
        if (hdr.x < 0) break;
        const int ab = item % NACC;
        if (hdr.y & kWsFirst) {
          // the accumulator must have been read out by the epilogue (its use item - NACC)
          if (!mbar_wait(aempty + ab, ((item / NACC) & 1) ^ 1, abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const unsigned abase = smem_u32(obuf);
        const unsigned dcol = tmem + (unsigned)(ab * MT * UN);
#pragma unroll 1
        for (int t = 0; t < MT; ++t) {
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const unsigned aoff = (unsigned)(t * 16 * L::SBO + ks * 2 * L::LBO);
            const unsigned boff = (unsigned)(ks * 2 * L::LBO);
            const uint64_t ahi = umma_sdesc(abase + (unsigned)L::ob_ahi + aoff, L::LBO, L::SBO);
            const uint64_t alo = umma_sdesc(abase + (unsigned)L::ob_alo + aoff, L::LBO, L::SBO);
            const uint64_t bhi = umma_sdesc(abase + (unsigned)L::ob_bhi + boff, L::LBO, L::SBO);
            const uint64_t blo = umma_sdesc(abase + (unsigned)L::ob_blo + boff, L::LBO, L::SBO);
            const unsigned first = (hdr.y & kWsFirst) && ks == 0;
            const unsigned d = dcol + (unsigned)(t * UN);
            umma_tf32(d, alo, bhi, idesc, first ? 0u : 1u);
            umma_tf32(d, ahi, blo, idesc, 1u);
            umma_tf32(d, ahi, bhi, idesc, 1u);
          }
        }
        umma_commit(oempty + ob);   // the operand buffer is free once these MMAs are done
        if (hdr.y & kWsLast) {
          acc_xy[ab] = hdr.z;
          mbar_arrive(afull + ab);   // window origin visible to the epilogue
          umma_commit(afull + ab);   // accumulator complete
          ++item;
        }
      }
      // tell the epilogue warps to stop: a phase of the next accumulator with the end marker
      const int ab = item % NACC;
      if (ok && mbar_wait(aempty + ab, ((item / NACC) & 1) ^ 1, abort_flag, err)) {
        acc_xy[ab] = -1;
        mbar_arrive(afull + ab);
        mbar_arrive(afull + ab);
      }
      // every MMA issued has completed before the tensor memory can be released (bounded wait
      // that ignores the abort flag)
      umma_commit(fin);
      volatile int never = 0;
      mbar_wait(fin, 0, &never, err);
    }
    __syncwarp();
  } else if (warp < 6) {
    // ------------------------------------------------------------------------------ epilogue
    const int q = warp & 3;   // tensor-memory lane quarter of this warp
    const int mode = (a.flags & AWG_GRID_FP64) ? 2 : (a.flags & AWG_GRID_KAHAN) ? 1 : 0;
    const size_t ystride = (size_t)a.N * P * 2;   // floats from one grid row to the next
    for (int item = 0;; ++item) {
      const int ab = item % NACC;
      if (!warp_wait(afull + ab, (item / NACC) & 1, abort_flag, err)) break;
      tc_fence_after();
      const int xy = acc_xy[ab];
      if (xy < 0) break;
      const int X0 = xy & 0xffff, Y0 = xy >> 16;
      const int ny = min(L::U, a.N - Y0);   // window rows inside the grid
      for (int t = 0; t < MT; ++t) {
        // row m = 128 t + 32 q + lane = (x, p, c): x = m / 2P, p = (m / 2) mod P, c = m mod 2
        const int m = 128 * t + 32 * q + lane;
        const int x = m / (2 * P), p = (m >> 1) % P, c = m & 1;
        const int gx = X0 + x;
        const bool col_ok = x < L::U && gx < a.N;
        const size_t e0 = (((size_t)Y0 * a.N + gx) * P + p) * 2 + c;   // float index of (gx, Y0, p, c)
        for (int y0 = 0; y0 < UN; y0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(ab * MT * UN + t * UN + y0), v);
          if (!col_ok || y0 >= ny) continue;
          const size_t e = e0 + (size_t)y0 * ystride;
          if (mode == 0) {
            float* g = a.grid + e;
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (y0 + i < ny && v[i] != 0.f) atomicAdd(g + (size_t)i * ystride, v[i]);
          } else if (mode == 1) {
            float* g = a.grid + e;
            float* glo = a.grid_lo + e;
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (y0 + i < ny && v[i] != 0.f) {
                const float old = atomicAdd(g + (size_t)i * ystride, v[i]);
                const float sum = old + v[i], bb = sum - old;
                const float er = (old - (sum - bb)) + (v[i] - bb);
                if (er != 0.f) atomicAdd(glo + (size_t)i * ystride, er);
              }
          } else {
            double* g = reinterpret_cast<double*>(a.grid) + e;
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (y0 + i < ny && v[i] != 0.f) atomicAdd(g + (size_t)i * ystride, (double)v[i]);
          }
        }
      }
      tc_fence_before();
      warp_arrive(aempty + ab);
    }
  } else {
    // ------------------------------------------------------------------------------ builders
    // A task (pixel-pol xp, K group kq) writes rows (x, p, 0) and (x, p, 1) over samples 2 kq and
    // 2 kq + 1; eight consecutive xp per K group, and lanes 4..7 of each eight write their c = 1
    // row first, so that the 16-byte stores of a warp fall in all eight bank groups.  A B task
    // (row y, K group kq) likewise with eight consecutive y.
    const int bt = tid - 6 * 32;   // 0 .. 32 NB_WARPS - 1
    constexpr int NBT = 32 * L::NB_WARPS;
    int q = 0;   // chunks handed to the MMA thread so far
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int s = k % D;
      unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
      if (!warp_wait(full + s, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      const int nsub = h.nst < 0 ? 1 : (h.nst + J - 1) / J;
      const int* pkv = reinterpret_cast<const int*>(sg + L::st_pk);
      const float2* fyv = reinterpret_cast<const float2*>(sg + L::st_fy);
      const float2* fxv = reinterpret_cast<const float2*>(sg + L::st_fx);
      const float2* wvv = reinterpret_cast<const float2*>(sg + L::st_wv);
      for (int sub = 0; sub < nsub; ++sub, ++q) {
        const int ob = q % NOB;
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        // the operand buffer is free once the MMAs that read it (chunk q - NOB) are done
        if (!warp_wait(oempty + ob, ((q / NOB) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        if (h.nst < 0) {
          if (bt == 0) *reinterpret_cast<int4*>(obuf + L::ob_hdr) = make_int4(-1, 0, 0, 0);
        } else {
          const int j0 = sub * J, n = min(J, h.nst - j0);
          const int fl = (sub == 0 ? (h.flags & kWsFirst) : 0) | (sub == nsub - 1 ? (h.flags & kWsLast) : 0);
          if (bt == 0) *reinterpret_cast<int4*>(obuf + L::ob_hdr) = make_int4(n, fl, h.xy, 0);
          for (int task = bt; task < L::UX * P * KQ; task += NBT) {
            const int xl = task & 7;
            const int kq = (task >> 3) % KQ;
            const int xp = (task / (8 * KQ)) * 8 + xl;
            const int x = xp / P, p = xp % P;
            float xr[2], xi[2];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int j = 2 * kq + h2;
              xr[h2] = 0.f;
              xi[h2] = 0.f;
              if (j < n) {
                const int tx = x - (pkv[j0 + j] & 0xff);
                if (tx >= 0 && tx < S) {
                  const float2 f = fxv[(j0 + j) * L::RS + tx];
                  const float2 w = wvv[(j0 + j) * P + p];
                  xr[h2] = f.x * w.x + f.y * w.y;   // conj(fx) w V
                  xi[h2] = f.x * w.y - f.y * w.x;
                }
              }
            }
            const int cfirst = (xl >> 2) & 1;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const int c = cc ^ cfirst;
              const int m = 2 * xp + c;
              // row c = 0: (Re X, Im X) per sample; row c = 1: (Im X, -Re X)
              const float e0 = c ? xi[0] : xr[0], e1 = c ? -xr[0] : xi[0];
              const float e2 = c ? xi[1] : xr[1], e3 = c ? -xr[1] : xi[1];
              float h0, h1, h2v, h3, l0, l1, l2, l3;
              tf32_split(e0, h0, l0);
              tf32_split(e1, h1, l1);
              tf32_split(e2, h2v, l2);
              tf32_split(e3, h3, l3);
              const size_t off = (size_t)(m % 8) * 16 + (size_t)(m / 8) * L::SBO + (size_t)kq * L::LBO;
              *reinterpret_cast<float4*>(obuf + L::ob_ahi + off) = make_float4(h0, h1, h2v, h3);
              *reinterpret_cast<float4*>(obuf + L::ob_alo + off) = make_float4(l0, l1, l2, l3);
            }
          }
          for (int task = b_first<L::UX * P * KQ, NBT>(bt); task < UN * KQ; task += NBT) {
            const int yl = task & 7;
            const int kq = (task >> 3) % KQ;
            const int y = (task / (8 * KQ)) * 8 + yl;
            float vv[4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int j = 2 * kq + h2;
              float br = 0.f, bi = 0.f;
              if (j < n) {
                const int ty = y - ((pkv[j0 + j] >> 8) & 0xff);
                if (ty >= 0 && ty < S) {
                  const float2 f = fyv[(j0 + j) * L::RS + ty];
                  br = f.x;
                  bi = f.y;
                }
              }
              vv[2 * h2] = br;
              vv[2 * h2 + 1] = bi;
            }
            float hi[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tf32_split(vv[i], hi[i], lo[i]);
            const size_t off = (size_t)(y % 8) * 16 + (size_t)(y / 8) * L::SBO + (size_t)kq * L::LBO;
            *reinterpret_cast<float4*>(obuf + L::ob_bhi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4*>(obuf + L::ob_blo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        fence_proxy_async_smem();   // the operands are read by the tensor cores (async proxy)
        warp_arrive(ofull + ob);
      }
      if (!ok) break;
      warp_arrive(empty + s);   // every chunk of the stage is built
      if (h.nst < 0) break;
    }
  }

  // every role has left its loop: release the tensor memory
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  __syncwarp();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)L::TCOLS));
}

template <int S, int P, int TILE, int J, int ST, int D, int NOB>
__global__ void __launch_bounds__(MmaNLayout<S, P, TILE, J, ST, D, NOB>::NT, 1)
    k_grid_mma_n(const GridArgs a, const int cls) {
  using L = MmaNLayout<S, P, TILE, J, ST, D, NOB>;
  constexpr int KS = L::KS, KQ = L::KQ, N = L::N, NACC = L::NACC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  int64_t* s_off = reinterpret_cast<int64_t*>(smem + L::off_soff);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* empty = full + D;
  uint64_t* ofull = full + 2 * D;
  uint64_t* oempty = ofull + NOB;
  uint64_t* afull = oempty + NOB;
  uint64_t* aempty = afull + NACC;
  uint64_t* fin = aempty + NACC;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::off_misc);
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(smem + L::off_misc + 16);
  int* acc_xy = reinterpret_cast<int*>(smem + L::off_misc + 32);
  unsigned long long* err = a.err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const bool off_cached = a.n_sep_off <= kSepOffCache;
  if (off_cached)
    for (int i = tid; i < a.n_sep_off; i += L::NT) s_off[i] = a.sep_off[i];
  const int64_t* offs = off_cached ? s_off : a.sep_off;
  if (tid == 0) {
    for (int d = 0; d < D; ++d) {
      mbar_init(full + d, 64);   // the producer lanes, then their copies
      mbar_init(empty + d, L::NB_WARPS);
    }
    for (int b = 0; b < NOB; ++b) {
      mbar_init(ofull + b, L::NB_WARPS);
      mbar_init(oempty + b, 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(afull + b, 2);
      mbar_init(aempty + b, 4);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
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
    mma_producer<S, P, TILE, ST, D, L>(a, cls, smem, full, empty, offs, abort_flag, err, lane);
  } else if (warp == 1) {
    // ------------------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr unsigned idesc = umma_idesc_tf32(128, N);
      int item = 0;
      bool ok = true;
      for (int q = 0;; ++q) {
        const int ob = q % NOB;
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        if (!mbar_wait(ofull + ob, (q / NOB) & 1, abort_flag, err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int4 hdr = *reinterpret_cast<const int4*>(obuf + L::ob_hdr);   // nst, flags, xy
        if (hdr.x < 0) break;
        const int ab = item % NACC;
        if (hdr.y & kWsFirst) {
          if (!mbar_wait(aempty + ab, ((item / NACC) & 1) ^ 1, abort_flag, err)) {
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
        const bool first = (hdr.y & kWsFirst) != 0;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const uint64_t o = (uint64_t)((ks * 2 * L::LBO) >> 4);   // start address field, 16-byte units
          umma_tf32(d, dal + o, dbh + o, idesc, (first && ks == 0) ? 0u : 1u);
          umma_tf32(d, dah + o, dbl + o, idesc, 1u);
          umma_tf32(d, dah + o, dbh + o, idesc, 1u);
        }
        umma_commit(oempty + ob);
        if (hdr.y & kWsLast) {
          acc_xy[ab] = hdr.z;
          mbar_arrive(afull + ab);
          umma_commit(afull + ab);
          ++item;
        }
      }
      const int ab = item % NACC;
      if (ok && mbar_wait(aempty + ab, ((item / NACC) & 1) ^ 1, abort_flag, err)) {
        acc_xy[ab] = -1;
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
    // Tensor-memory lane m = 32 q + lane holds row (x, c) = (m / 2, m mod 2) of the window, one
    // column per (y, p).  Lanes 2i and 2i + 1 swap half of each 16 columns so that each holds both
    // parts of its complex values: lane c keeps columns with bit 1 equal to c, i.e. pols p, p + 1
    // of a pixel (P >= 2; one 16-byte atomic) or rows y, y + 1 (P = 1).
    const int q = warp & 3;
    const int mode = (a.flags & AWG_GRID_FP64) ? 2 : (a.flags & AWG_GRID_KAHAN) ? 1 : 0;
    const size_t ystride = (size_t)a.N * P * 2;
    const int m = 32 * q + lane, x = m >> 1, c = m & 1;
    for (int item = 0;; ++item) {
      const int ab = item % NACC;
      if (!warp_wait(afull + ab, (item / NACC) & 1, abort_flag, err)) break;
      tc_fence_after();
      const int xy = acc_xy[ab];
      if (xy < 0) break;
      const int X0 = xy & 0xffff, Y0 = xy >> 16;
      const int gx = X0 + x;
      const bool col_ok = x < L::U && gx < a.N;
      const int ny = min(L::U, a.N - Y0);
      const size_t ebase = ((size_t)Y0 * a.N + gx) * P * 2;   // float index of (gx, Y0, pol 0, Re)
      for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(ab * N + n0), v);
        float re[8], im[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int k0 = (t >> 1) * 4 + (t & 1);   // t-th column kept by an even lane
          const float send = c ? v[k0] : v[k0 + 2];
          const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
          const float own = c ? v[k0 + 2] : v[k0];
          re[t] = c ? recv : own;
          im[t] = c ? own : recv;
        }
        if (!col_ok) continue;
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
          const int n = n0 + (t >> 1) * 4 + 2 * c;   // even column: (y, p) with p even, or row y
          if constexpr (P >= 2) {
            const int y = n / P, p = n % P;
            if (y < ny)
              mma_flush4(a.grid, a.grid_lo, ebase + (size_t)y * ystride + 2 * p, mode,
                         make_float4(re[t], im[t], re[t + 1], im[t + 1]));
          } else {
            if (n < ny) mma_flush2(a.grid, a.grid_lo, ebase + (size_t)n * ystride, mode, make_float2(re[t], im[t]));
            if (n + 1 < ny)
              mma_flush2(a.grid, a.grid_lo, ebase + (size_t)(n + 1) * ystride, mode, make_float2(re[t + 1], im[t + 1]));
          }
        }
      }
      tc_fence_before();
      warp_arrive(aempty + ab);
    }
  } else {
    // ------------------------------------------------------------------------------ builders
    // A task (row m = (x, c), K group kq) holds samples 2 kq, 2 kq + 1 of the conjugated x factor:
    // (Re, Im) of fx in row c = 0 and (-Im, Re) in row c = 1.  A B task (row n = (y, p)) holds
    // conj(fy) w V.  Eight consecutive rows per K group, so that the 16-byte stores of a warp fall
    // in all eight bank groups.
    const int bt = tid - 6 * 32;
    constexpr int NBT = 32 * L::NB_WARPS;
    // A rows (x, c) with x >= U are zero for every sample (first taps lie in [0, TILE)): written
    // once here in every operand buffer and never again.  The MMA thread reads a buffer only after
    // every builder warp has arrived on it, so these stores come first.
    constexpr int AR = 2 * L::U;   // A rows that are built per chunk
    static_assert(AR % 8 == 0, "A rows are built in groups of eight");
    for (int b = 0; b < NOB; ++b) {
      unsigned char* obuf = smem + L::off_ob + (size_t)b * L::ob_bytes;
      for (int i = AR * KQ + bt; i < 128 * KQ; i += NBT) {
        const int kq = i % KQ, m = i / KQ;
        const size_t off = (size_t)(m % 8) * 16 + (size_t)(m / 8) * L::SBO + (size_t)kq * L::LBO;
        *reinterpret_cast<float4*>(obuf + L::ob_ahi + off) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(obuf + L::ob_alo + off) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    int q = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int s = k % D;
      unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
      if (!warp_wait(full + s, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      const int nsub = h.nst < 0 ? 1 : (h.nst + J - 1) / J;
      const int* pkv = reinterpret_cast<const int*>(sg + L::st_pk);
      const float2* fyv = reinterpret_cast<const float2*>(sg + L::st_fy);
      const float2* fxv = reinterpret_cast<const float2*>(sg + L::st_fx);
      const float2* wvv = reinterpret_cast<const float2*>(sg + L::st_wv);
      for (int sub = 0; sub < nsub; ++sub, ++q) {
        const int ob = q % NOB;
        unsigned char* obuf = smem + L::off_ob + (size_t)ob * L::ob_bytes;
        if (!warp_wait(oempty + ob, ((q / NOB) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        if (h.nst < 0) {
          if (bt == 0) *reinterpret_cast<int4*>(obuf + L::ob_hdr) = make_int4(-1, 0, 0, 0);
        } else {
          const int j0 = sub * J, n = min(J, h.nst - j0);
          const int fl = (sub == 0 ? (h.flags & kWsFirst) : 0) | (sub == nsub - 1 ? (h.flags & kWsLast) : 0);
          if (bt == 0) *reinterpret_cast<int4*>(obuf + L::ob_hdr) = make_int4(n, fl, h.xy, 0);
#pragma unroll 4
          for (int task = bt; task < AR * KQ; task += NBT) {
            const int kq = (task >> 3) % KQ;
            const int m = (task / (8 * KQ)) * 8 + (task & 7);
            const int x = m >> 1, c = m & 1;
            float e[4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int j = 2 * kq + h2;
              float fr = 0.f, fi = 0.f;
              if (j < n) {
                const int tx = x - (pkv[j0 + j] & 0xff);
                if (tx >= 0 && tx < S) {
                  const float2 f = fxv[(j0 + j) * L::RS + tx];
                  fr = f.x;
                  fi = f.y;
                }
              }
              e[2 * h2] = c ? -fi : fr;
              e[2 * h2 + 1] = c ? fr : fi;
            }
            float hi[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tf32_split(e[i], hi[i], lo[i]);
            const size_t off = (size_t)(m % 8) * 16 + (size_t)(m / 8) * L::SBO + (size_t)kq * L::LBO;
            *reinterpret_cast<float4*>(obuf + L::ob_ahi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4*>(obuf + L::ob_alo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
#pragma unroll 4
          for (int task = b_first<AR * KQ, NBT>(bt); task < N * KQ; task += NBT) {
            const int kq = (task >> 3) % KQ;
            const int nn = (task / (8 * KQ)) * 8 + (task & 7);
            const int y = nn / P, p = nn % P;
            float e[4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int j = 2 * kq + h2;
              float br = 0.f, bi = 0.f;
              if (j < n) {
                const int ty = y - ((pkv[j0 + j] >> 8) & 0xff);
                if (ty >= 0 && ty < S) {
                  const float2 f = fyv[(j0 + j) * L::RS + ty];
                  const float2 w = wvv[(j0 + j) * P + p];
                  br = f.x * w.x + f.y * w.y;   // conj(fy) w V
                  bi = f.x * w.y - f.y * w.x;
                }
              }
              e[2 * h2] = br;
              e[2 * h2 + 1] = bi;
            }
            float hi[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tf32_split(e[i], hi[i], lo[i]);
            const size_t off = (size_t)(nn % 8) * 16 + (size_t)(nn / 8) * L::SBO + (size_t)kq * L::LBO;
            *reinterpret_cast<float4*>(obuf + L::ob_bhi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4*>(obuf + L::ob_blo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
        fence_proxy_async_smem();
        warp_arrive(ofull + ob);
      }
      if (!ok) break;
      warp_arrive(empty + s);
      if (h.nst < 0) break;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  __syncwarp();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)L::TCOLS));
}

// Tensor-core configuration per exact support and pol count: the tile of first-tap positions
// (window side S + TILE - 1 at or just below a multiple of 16, so that little of the padded window
// is waste; it depends on S alone, the plan bins by it), samples per MMA chunk and per producer
// stage, stages and operand buffers.  Two operand buffers cover the MMAs of a chunk (they take far
// less time than building the next one); the rest of the shared memory goes to stages, whose
// samples in flight hide the latency of the factor-row copies.
struct MmaCfg {
  int S, P, tile, j, st, d, nob;
};
// pols in M (k_grid_mma): windows wider than one 128-row tile of (x, re/im) rows
constexpr MmaCfg kMmaCfg[3] = {{64, 1, 9, 8, 32, 2, 3}, {64, 2, 9, 8, 32, 3, 2}, {64, 4, 9, 8, 16, 2, 2}};
// pols in N (k_grid_mma_n): windows of side <= 64
constexpr MmaCfg kMmaNCfg[21] = {
    {8, 1, 9, 16, 32, 8, 2},   {8, 2, 9, 16, 32, 8, 2},   {8, 4, 9, 16, 32, 8, 2},   {16, 1, 17, 16, 32, 8, 2},
    {16, 2, 17, 16, 32, 8, 2}, {16, 4, 17, 16, 32, 8, 2}, {24, 1, 9, 16, 32, 8, 2},  {24, 2, 9, 16, 32, 8, 2},
    {24, 4, 9, 16, 32, 6, 2},  {32, 1, 17, 16, 32, 7, 2}, {32, 2, 17, 16, 32, 6, 2}, {32, 4, 17, 16, 32, 3, 2},
    {40, 1, 9, 16, 32, 6, 2},  {40, 2, 9, 16, 32, 5, 2},  {40, 4, 9, 16, 32, 2, 2},  {48, 1, 17, 16, 32, 4, 2},
    {48, 2, 17, 16, 32, 3, 2}, {48, 4, 17, 8, 32, 4, 2},  {56, 1, 9, 16, 32, 4, 2},  {56, 2, 9, 16, 32, 3, 2},
    {56, 4, 9, 8, 32, 4, 2},
};
constexpr MmaCfg mma_cfg(int S, int P) {
  for (const MmaCfg& e : kMmaCfg)
    if (e.S == S && e.P == P) return e;
  return MmaCfg{S, P, 0, 0, 0, 0, 0};
}
constexpr MmaCfg mma_n_cfg(int S, int P) {
  for (const MmaCfg& e : kMmaNCfg)
    if (e.S == S && e.P == P) return e;
  return MmaCfg{S, P, 0, 0, 0, 0, 0};
}

template <class Kern>
awg_status launch_grid_mma(Kern kern, int& ready, int nt, size_t alloc, const GridArgs& a, int slot, int sms,
                           cudaStream_t st) {
  if (!ready) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)alloc));
    int bps = 0;
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, nt, alloc));
    if (bps != 1) return set_error(AWG_ERR_CUDA, "tensor-core gridding kernel must hold an SM alone");
    ready = 1;
  }
  kern<<<sms, nt, alloc, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

template <int S, int P>
awg_status run_grid_mma(const GridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr int T = exact_cfg(S, 3).tile;
  static int ready = 0;
  if constexpr (T + S - 1 <= 64) {
    constexpr MmaCfg c = mma_n_cfg(S, P);
    static_assert(c.tile == T, "the plan bins candidate 3 by this tile");
    using L = MmaNLayout<S, P, c.tile, c.j, c.st, c.d, c.nob>;
    static_assert(L::alloc <= 227 * 1024, "tensor-core gridding stages do not fit");
    return launch_grid_mma(k_grid_mma_n<S, P, c.tile, c.j, c.st, c.d, c.nob>, ready, L::NT, L::alloc, a, slot, sms,
                           st);
  } else {
    constexpr MmaCfg c = mma_cfg(S, P);
    static_assert(c.tile == T, "the plan bins candidate 3 by this tile");
    using L = MmaGridLayout<S, P, c.tile, c.j, c.st, c.d, c.nob>;
    static_assert(L::alloc <= 227 * 1024, "tensor-core gridding stages do not fit");
    return launch_grid_mma(k_grid_mma<S, P, c.tile, c.j, c.st, c.d, c.nob>, ready, L::NT, L::alloc, a, slot, sms, st);
  }
}

#define AWG_FOR_MMA(M) M(8, 1) M(8, 2) M(8, 4) M(16, 1) M(16, 2) M(16, 4) M(24, 1) M(24, 2) M(24, 4) M(32, 1) M(32, 2) M(32, 4) \
  M(40, 1) M(40, 2) M(40, 4) M(48, 1) M(48, 2) M(48, 4) M(56, 1) M(56, 2) M(56, 4) M(64, 1) M(64, 2) M(64, 4)
#define AWG_DECLARE_GRID_MMA(S, P) extern template awg_status run_grid_mma<S, P>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_MMA(S, P) template awg_status run_grid_mma<S, P>(const GridArgs&, int, int, cudaStream_t);

}  // namespace awg
