// Warp-specialised gridding and degridding with separable rank-1 CF records on the exact
// supports (the W-projection schedule): the arithmetic of resample_sep.cuh, with the per-chunk
// CTA barriers replaced by a ring of shared-memory stages handed over on mbarriers.
//
// Roles (one persistent CTA pulls work items of one support from its queue):
//  * warp 0, the producer, walks the CTA's items chunk by chunk.  It keeps the records of the next
//    two chunks and the visibilities, weights and phasors of the next one in registers (loads
//    issued ahead), and for each chunk writes the packed first-tap positions, w V times the phasor
//    (gridding) or the output rows and phasors (degridding) into a free stage and moves each
//    sample's two factor rows fx[ox][.], fy[oy][.] into it with one TMA bulk copy per row, whose
//    bytes complete the stage's barrier.
//  * the consumer warps own the taps by residue as in resample_sep.cuh (thread: column residue rx,
//    rows ry0 + k G) and run only the multiply-add loop over the samples of each stage; a stage is
//    released when every consumer thread has read it.
//  * gridding: the consumers accumulate an item in one of NWIN shared windows.  A window pixel is
//    only ever touched by the thread whose residues it has, so at the end of the item each thread
//    adds its own pixels to the grid (one vector atomic per non-zero pixel) and zeroes them, with
//    no barrier; a window is reused NWIN items later, once every thread has flushed it.
//  * degridding: warp 1 reduces.  The producer loads each item's grid window with one TMA tile
//    copy (cp.async.bulk.tensor) into one of NWIN windows; the consumers leave one warp-reduced
//    value per lane and batch of every stage, and the reduce warp adds the consumer warps' values,
//    applies the phasor and writes the visibilities.
// No CTA-wide barrier runs after the set-up; every hand-off is an mbarrier phase, every wait is
// bounded (ws_sync.cuh).
#pragma once

#include <type_traits>

#include "resample_sep.cuh"
#include "ws_sync.cuh"

namespace awg {

// Flags of a stage header.
constexpr int kWsFirst = 1, kWsLast = 2;

struct __align__(16) WsHeader {
  int nst;     // samples in the stage; -1: no more work
  int flags;   // kWsFirst / kWsLast of the item
  int xy;      // X0 | Y0 << 16 of the item's window
  int nr;      // runs of equal first-tap position in the stage
};

// The runs of a chunk: samples [rs[r], rs[r + 1]) share the packed first-tap position rpk[r] (the
// samples of an item are sorted by first tap).  Written by the producer warp from the packed
// positions of its lanes (lane j < nst holds sample j's); returns the number of runs.
__device__ __forceinline__ int ws_runs(int pk, int nst, int lane, int* rs, int* rpk) {
  const int up = __shfl_up_sync(0xffffffffu, pk, 1);
  const bool start = lane < nst && (lane == 0 || up != pk);
  const unsigned m = __ballot_sync(0xffffffffu, start);
  const int nr = __popc(m);
  if (start) {
    const int r = __popc(m & ((1u << lane) - 1u));
    rs[r] = lane;
    rpk[r] = pk;
  }
  if (lane == 0) rs[nr] = nst;
  return nr;
}

// Column residue and first row of consumer thread t of NC warps (as tap_owner): a warp covers 8
// consecutive columns x 4 row groups when the columns split into blocks of 8 that the warps tile,
// else rx = t mod S, ry0 = t div S.
template <int S, int G>
__device__ __forceinline__ void ws_owner(int t, int& rx, int& ry0) {
  constexpr int NC = S * G / 32;
  if constexpr (S % 8 == 0 && G % 4 == 0 && NC % (S / 8) == 0) {
    const int lane = t & 31, w = t >> 5;
    rx = (w % (S / 8)) * 8 + (lane & 7);
    ry0 = (w / (S / 8)) * 4 + (lane >> 3);
  } else {
    rx = t % S;
    ry0 = t / S;
  }
}

constexpr size_t ws_al16(size_t b) { return (b + 15) & ~(size_t)15; }
constexpr size_t ws_al1k(size_t b) { return (b + 1023) & ~(size_t)1023; }

// The producer's walk over the CTA's items: descriptor of one chunk.
struct WsChunk {
  int start, nst, xy, flags;
  bool valid;
};

// The producer's walk over the items a CTA takes from its queue, with the next item fetched ahead:
// the queue atomic is issued when an item is taken, its result is read and the next item's
// descriptor loaded one chunk later, and both are ready long before the current item ends (a
// wait happens only when an item has a single chunk).  All lanes of the producer warp keep the
// same state; the atomic's result lives in lane 0.
struct WsItemWalker {
  int begin, end, cls, tile, st;
  int32_t* queue;
  const WorkItem* items;
  WorkItem cur, nxt;
  int c, nch;        // next chunk of the current item, chunks of the item
  bool cur_valid;
  int q_raw;         // lane 0: the queue position the atomic returned
  int q_state;       // 1: atomic issued, 2: next item loaded, 3: queue exhausted

  __device__ __forceinline__ void issue() {
    if ((threadIdx.x & 31) == 0) q_raw = atomicAdd(queue + cls, 1);
    q_state = 1;
  }
  __device__ __forceinline__ void advance() {
    if (q_state == 1) {
      const int idx = begin + __shfl_sync(0xffffffffu, q_raw, 0);
      if (idx < end) {
        nxt = items[idx];
        q_state = 2;
      } else {
        q_state = 3;
      }
    }
  }
  __device__ __forceinline__ void take() {
    advance();
    if (q_state == 2) {
      cur = nxt;
      cur_valid = true;
      c = 0;
      nch = (cur.count + st - 1) / st;
      issue();
    } else {
      cur_valid = false;
    }
  }
  __device__ __forceinline__ void init(int b, int e, int cl, int t, int stage, int32_t* q, const WorkItem* it) {
    begin = b;
    end = e;
    cls = cl;
    tile = t;
    st = stage;
    queue = q;
    items = it;
    cur_valid = false;
    issue();
    take();
  }
  __device__ __forceinline__ WsChunk next() {
    WsChunk d{0, 0, 0, 0, false};
    if (cur_valid && c >= nch) take();
    if (!cur_valid) return d;
    d.start = cur.start + c * st;
    d.nst = min(st, cur.count - c * st);
    d.xy = (cur.tile_x * tile) | ((cur.tile_y * tile) << 16);
    d.flags = (c == 0 ? kWsFirst : 0) | (c == nch - 1 ? kWsLast : 0);
    d.valid = true;
    ++c;
    advance();   // one step of the fetch-ahead per chunk
    return d;
  }
};

// Record of sample `lane` of a chunk (a zero record past its end).
__device__ __forceinline__ SampleRec ws_load_rec(const SampleRec* rec, const WsChunk& d, int lane) {
  SampleRec r{};
  if (d.valid && lane < d.nst) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(rec + d.start + lane));
    r = *reinterpret_cast<const SampleRec*>(&v);
  }
  return r;
}

// Factor-row offsets (in complex values) of a record: fx[ox][.] and fy[oy][.] of its CF term.
template <int S>
__device__ __forceinline__ void ws_rows(const int64_t* offs, int64_t cf_shift, int OS, const SampleRec& rc,
                                        long long& fxo, long long& fyo) {
  const long long base = offs[cf_shift + rc.cf];
  fxo = base + (long long)rc.ox * S;
  fyo = base + (long long)(OS + 1) * S + (long long)rc.oy * S;
}

// Visibilities, weights and phasor of one sample, loaded by the producer a chunk ahead.
template <int P>
struct WsVis {
  float2 v[P];
  float w[P];
  float2 ph;
};

template <int P>
__device__ __forceinline__ WsVis<P> ws_load_vis(const GridArgs& a, const WsChunk& d, const SampleRec& rc, int lane) {
  WsVis<P> x;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    x.v[p] = make_float2(0.f, 0.f);
    x.w[p] = 0.f;
  }
  x.ph = make_float2(1.f, 0.f);
  if (d.valid && lane < d.nst) {
    const size_t s = (size_t)rc.src;
    if constexpr (P == 4) {
      const float4 a0 = __ldg(reinterpret_cast<const float4*>(a.vis + s * 8));
      const float4 a1 = __ldg(reinterpret_cast<const float4*>(a.vis + s * 8 + 4));
      const float4 ww = __ldg(reinterpret_cast<const float4*>(a.weight + s * 4));
      x.v[0] = make_float2(a0.x, a0.y);
      x.v[1] = make_float2(a0.z, a0.w);
      x.v[2] = make_float2(a1.x, a1.y);
      x.v[3] = make_float2(a1.z, a1.w);
      x.w[0] = ww.x;
      x.w[1] = ww.y;
      x.w[2] = ww.z;
      x.w[3] = ww.w;
    } else if constexpr (P == 2) {
      const float4 a0 = __ldg(reinterpret_cast<const float4*>(a.vis + s * 4));
      const float2 ww = __ldg(reinterpret_cast<const float2*>(a.weight + s * 2));
      x.v[0] = make_float2(a0.x, a0.y);
      x.v[1] = make_float2(a0.z, a0.w);
      x.w[0] = ww.x;
      x.w[1] = ww.y;
    } else {
      x.v[0] = __ldg(reinterpret_cast<const float2*>(a.vis) + s);
      x.w[0] = __ldg(a.weight + s);
    }
    if (a.phasor) x.ph = __ldg(a.phasor + rc.src);
  }
  return x;
}

// ------------------------------------------------------------------------------------ gridding

template <int S, int P, int G, int TILE, int ST, int D, int NWIN>
struct WsGridLayout {
  static_assert(S % G == 0 && (S * G) % 32 == 0, "row groups must divide S and fill whole warps");
  static_assert(S % 2 == 0, "factor rows move in 16-byte units");
  static constexpr int NC = S * G / 32;          // consumer warps
  static constexpr int NT = 32 * (NC + 1);       // + the producer
  static constexpr int R = S / G;                // rows per consumer thread
  static constexpr int U = TILE + S - 1;
  static constexpr int UU = U * U;
  static constexpr size_t win_bytes = ws_al16((size_t)UU * P * 8);   // pol-planar float2 [P][U][U]
  // a stage: header, runs (starts, positions), fy rows twice over (fy[t] at t and t + S, so that a
  // thread's rows sit at fixed offsets from S - my), fx rows, w V (times the phasor) per pol
  static constexpr size_t st_rs = 16;
  static constexpr size_t st_rpk = st_rs + ws_al16(4 * (ST + 1));
  static constexpr size_t st_fy = st_rpk + ws_al16(4 * ST);
  static constexpr size_t st_fx = st_fy + (size_t)ST * 2 * S * 8;
  static constexpr size_t st_wv = st_fx + (size_t)ST * S * 8;
  static constexpr size_t stage_bytes = ws_al16(st_wv + (size_t)ST * P * 8);
  static constexpr size_t off_stage = NWIN * win_bytes;
  static constexpr size_t off_bar = off_stage + D * stage_bytes;
  static constexpr size_t off_misc = off_bar + 8 * (2 * D + NWIN);
  static constexpr size_t off_soff = ws_al16(off_misc + 16);   // int64 [kSepOffCache]
  static constexpr size_t bytes = off_soff + 8 * (size_t)kSepOffCache;
  static constexpr size_t alloc = bytes + 1024;   // the layout starts at the first 1024-byte boundary
};

template <int S, int P, int G, int TILE, int ST, int D, int NWIN, int MINB>
__global__ void __launch_bounds__(WsGridLayout<S, P, G, TILE, ST, D, NWIN>::NT, MINB)
    k_grid_ws(const GridArgs a, const int cls) {
  using L = WsGridLayout<S, P, G, TILE, ST, D, NWIN>;
  constexpr int NC = L::NC, R = L::R, U = L::U, UU = L::UU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  int64_t* s_off = reinterpret_cast<int64_t*>(smem + L::off_soff);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* empty = full + D;
  uint64_t* wdone = full + 2 * D;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::off_misc);
  unsigned long long* err = a.err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const bool off_cached = a.n_sep_off <= kSepOffCache;
  if (off_cached)
    for (int i = tid; i < a.n_sep_off; i += L::NT) s_off[i] = a.sep_off[i];
  const int64_t* offs = off_cached ? s_off : a.sep_off;
  if (tid == 0) {
    for (int d = 0; d < D; ++d) {
      mbar_init(full + d, 32);
      mbar_init(empty + d, NC * 32);
    }
    for (int w = 0; w < NWIN; ++w) mbar_init(wdone + w, NC * 32);
    *abort_flag = 0;
    mbar_fence_init();
  }
  {
    float2* win = reinterpret_cast<float2*>(smem);
    for (int i = tid; i < NWIN * (int)(L::win_bytes / 8); i += L::NT) win[i] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------------------------------ producer
    double wsum[P];
#pragma unroll
    for (int p = 0; p < P; ++p) wsum[p] = 0.0;
    WsItemWalker walk;
    walk.init(a.class_range[cls], a.class_range[cls + 1], cls, TILE, ST, a.queue, a.items);
    const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
    // loads run ahead of their use: the records three chunks, the visibilities two
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
      if (!mbar_wait(empty + s, ((k / D) & 1) ^ 1, abort_flag, err)) {
        ok = false;
        break;
      }
      const int X0 = d0.xy & 0xffff, Y0 = d0.xy >> 16;
      const int pk = (r0.p0x - X0) | ((r0.p0y - Y0) << 8) | ((r0.p0x % S) << 16) | ((r0.p0y % S) << 24);
      const int nr = ws_runs(pk, d0.nst, lane, reinterpret_cast<int*>(sg + L::st_rs),
                             reinterpret_cast<int*>(sg + L::st_rpk));
      if (lane < d0.nst) {
        long long fxo, fyo;
        ws_rows<S>(offs, a.cf_shift, a.OS, r0, fxo, fyo);
        fence_proxy_async_smem();   // the consumers' reads of this stage come before the copies
        bulk_load(sg + L::st_fx + (size_t)lane * S * 8, sep2 + fxo, S * 8, full + s);
        bulk_load(sg + L::st_fy + (size_t)lane * 2 * S * 8, sep2 + fyo, S * 8, full + s);
        bulk_load(sg + L::st_fy + (size_t)lane * 2 * S * 8 + S * 8, sep2 + fyo, S * 8, full + s);
        float2 o[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const float xr = x0.w[p] * x0.v[p].x, xi = x0.w[p] * x0.v[p].y;
          o[p] = make_float2(xr * x0.ph.x - xi * x0.ph.y, xr * x0.ph.y + xi * x0.ph.x);
        }
        float2* dst = reinterpret_cast<float2*>(sg + L::st_wv) + lane * P;
        if constexpr (P % 2 == 0) {
#pragma unroll
          for (int q = 0; q < P / 2; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(o[2 * q].x, o[2 * q].y, o[2 * q + 1].x, o[2 * q + 1].y);
        } else {
          dst[0] = o[0];
        }
        if (a.rank == 1 || r0.cf % a.rank == 0) {   // term 0 of a sample adds its weights
#pragma unroll
          for (int p = 0; p < P; ++p) wsum[p] += (double)x0.w[p];
        }
      }
      if (lane == 0) *reinterpret_cast<WsHeader*>(sg) = WsHeader{d0.nst, d0.flags, d0.xy, nr};
      // hand over: lane 0 announces the bytes of the chunk's row copies; with the 32 arrivals and
      // those bytes the stage is full
      if (!(a.withhold && k == 0)) {
        if (lane == 0) mbar_arrive_expect_tx(full + s, (unsigned)(d0.nst * 3 * S * 8));
        else mbar_arrive(full + s);
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
    if (ok && mbar_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
      if (lane == 0) *reinterpret_cast<WsHeader*>(smem + L::off_stage + (size_t)(k % D) * L::stage_bytes) =
          WsHeader{-1, 0, 0, 0};
      mbar_arrive(full + k % D);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      double v = wsum[p];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && v != 0.0 && a.sumwt) atomicAdd(a.sumwt + p, v);
    }
  } else {
    // ------------------------------------------------------------------------------ consumers
    const int ct = tid - 32;
    int rx, ry0;
    ws_owner<S, G>(ct, rx, ry0);
    float2 acc[R][P];
    int curY[R], Y[R];
    int curX = -1, tx = 0, rowoff = 0, prev_pk = -1, prev_row = -1;
    int X0 = 0, Y0 = 0;
    float2* win = reinterpret_cast<float2*>(smem);
    int ic = 0;
#pragma unroll
    for (int kk = 0; kk < R; ++kk) {
      curY[kk] = -1;
      Y[kk] = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) acc[kk][p] = make_float2(0.f, 0.f);
    }
    for (int k = 0;; ++k) {
      const int s = k % D;
      unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
      if (!mbar_wait(full + s, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      if (h.nst < 0) break;
      const int w = ic % NWIN;
      if (h.flags & kWsFirst) {
        // a new item: its window must have been flushed by every thread
        if (!mbar_wait(wdone + w, ((ic / NWIN) & 1) ^ 1, abort_flag, err)) break;
        win = reinterpret_cast<float2*>(smem + (size_t)w * L::win_bytes);
        X0 = h.xy & 0xffff;
        Y0 = h.xy >> 16;
        curX = -1;
        prev_pk = -1;
        prev_row = -1;
      }
      const int* rsv = reinterpret_cast<const int*>(sg + L::st_rs);
      const int* rpkv = reinterpret_cast<const int*>(sg + L::st_rpk);
      const float2* fyb = reinterpret_cast<const float2*>(sg + L::st_fy);
      const float2* fxb = reinterpret_cast<const float2*>(sg + L::st_fx);
      const float2* wvb = reinterpret_cast<const float2*>(sg + L::st_wv);
      for (int r = 0; r < h.nr; ++r) {
        const int pk = rpkv[r];
        if (pk != prev_pk) {   // the first tap moved (once per run, the same in every consumer thread)
          prev_pk = pk;
          const int dx = pk & 0xff, mx = (pk >> 16) & 0xff;
          const int row = pk & 0xff00ff00;
          bool row_changed = false;
          if (row != prev_row) {
            prev_row = row;
            const int dy = (pk >> 8) & 0xff, my = (pk >> 24) & 0xff;
            rowoff = S - my + ry0;   // fy of row ry0 + kk G at rowoff + kk G of the doubled row
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
              int t = ry0 + kk * G - my;
              t += (t < 0) ? S : 0;
              Y[kk] = dy + t;
            }
            row_changed = true;
          }
          tx = rx - mx;
          tx += (tx < 0) ? S : 0;
          const int X = dx + tx;
          if (X != curX || row_changed) {
            const bool xchg = X != curX;
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
              if (xchg || Y[kk] != curY[kk]) {
                if (curY[kk] >= 0) {
#pragma unroll
                  for (int p = 0; p < P; ++p) {
                    float2* t = win + p * UU + curY[kk] * U + curX;
                    t->x += acc[kk][p].x;
                    t->y += acc[kk][p].y;
                    acc[kk][p] = make_float2(0.f, 0.f);
                  }
                }
                curY[kk] = Y[kk];
              }
            }
            curX = X;
          }
        }
        const int j1 = rsv[r + 1];
        const float2* fxp = fxb + rsv[r] * S + tx;
        const float2* fyp = fyb + rsv[r] * 2 * S + rowoff;
        const float2* wvp = wvb + rsv[r] * P;
        for (int j = rsv[r]; j < j1; ++j, fxp += S, fyp += 2 * S, wvp += P) {
          // alpha_p = conj(fx) w V_p for this thread's column
          const float2 fx = *fxp;
          float2 al[P];
          load_pols<P>(wvp, al);
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const float ar = al[p].x, ai = al[p].y;
            al[p] = make_float2(fx.x * ar + fx.y * ai, fx.x * ai - fx.y * ar);
          }
#pragma unroll
          for (int kk = 0; kk < R; ++kk) {
            const float2 f = fyp[kk * G];
#pragma unroll
            for (int p = 0; p < P; ++p) {   // acc += conj(fy) alpha
              acc[kk][p].x = fmaf(f.x, al[p].x, fmaf(f.y, al[p].y, acc[kk][p].x));
              acc[kk][p].y = fmaf(f.x, al[p].y, fmaf(-f.y, al[p].x, acc[kk][p].y));
            }
          }
        }
      }
      mbar_arrive(empty + s);
      if (h.flags & kWsLast) {
        // the item is complete: registers into the window, then this thread's own window pixels
        // (absolute column = rx, rows = ry0 + kk G modulo S) to the grid
#pragma unroll
        for (int kk = 0; kk < R; ++kk) {
          if (curY[kk] >= 0) {
#pragma unroll
            for (int p = 0; p < P; ++p) {
              float2* t = win + p * UU + curY[kk] * U + curX;
              t->x += acc[kk][p].x;
              t->y += acc[kk][p].y;
              acc[kk][p] = make_float2(0.f, 0.f);
            }
          }
          curY[kk] = -1;
        }
        const int xs = (rx - X0 % S + S) % S;
        for (int X = xs; X < U; X += S) {
#pragma unroll
          for (int kk = 0; kk < R; ++kk) {
            const int ys = (ry0 + kk * G - Y0 % S + S) % S;
            for (int Yw = ys; Yw < U; Yw += S) {
              float2 v[P];
              bool nz = false;
#pragma unroll
              for (int p = 0; p < P; ++p) {
                v[p] = win[p * UU + Yw * U + X];
                nz |= (v[p].x != 0.f) || (v[p].y != 0.f);
              }
              if (nz) {
#pragma unroll
                for (int p = 0; p < P; ++p) win[p * UU + Yw * U + X] = make_float2(0.f, 0.f);
                const int gy = Y0 + Yw, gx = X0 + X;
                if (gy < a.N && gx < a.N) flush_pixel<P>(a, ((size_t)gy * a.N + gx) * P, v);
              }
            }
          }
        }
        mbar_arrive(wdone + w);
        ++ic;
      }
    }
  }
}

// ---------------------------------------------------------------------------------- degridding

template <int S, int P, int G, int TILE, int ST, int D, int NWIN>
struct WsDegridLayout {
  static_assert(S % G == 0 && (S * G) % 32 == 0, "row groups must divide S and fill whole warps");
  static_assert(S % 2 == 0, "factor rows move in 16-byte units");
  static constexpr int NC = S * G / 32;
  static constexpr int NT = 32 * (NC + 2);        // + producer + reduce warp
  static constexpr int R = S / G;
  static constexpr int U = TILE + S - 1;
  static constexpr int B = 32 / (2 * P);          // samples per butterfly batch
  static constexpr int NB = (ST + B - 1) / B;     // batches per stage
  // window as the TMA tile lands: P >= 2: [U][U][P] c64 (3-D box (2P, U, U)); P = 1: rows of UB
  // pixels (2-D box (2 UB, U)).  A P = 1 box starts at an even pixel (its x coordinate, 8 bytes a
  // pixel, must be a multiple of 16 bytes): with an odd tile the window origin X0 may be odd, and
  // the box then starts one pixel early (XA = 1 extra column) and the window sits at X0 & 1 in it.
  // UB is U + XA rounded up to even, so that a box row is a whole number of 16-byte units.
  static constexpr int XA = (P == 1 && TILE % 2 == 1) ? 1 : 0;
  static constexpr int UB = (P == 1) ? ((U + XA + 1) & ~1) : U;
  static_assert(P != 1 || 2 * UB <= 256, "a TMA box side holds at most 256 elements");
  static constexpr unsigned box_bytes = (unsigned)U * UB * P * 8;
  static constexpr size_t win_bytes = ws_al1k(box_bytes);
  static constexpr size_t st_rs = 16;
  static constexpr size_t st_rpk = st_rs + ws_al16(4 * (ST + 1));
  static constexpr size_t st_fy = st_rpk + ws_al16(4 * ST);   // fy rows twice over, as for gridding
  static constexpr size_t st_fx = st_fy + (size_t)ST * 2 * S * 8;
  static constexpr size_t st_src = st_fx + (size_t)ST * S * 8;
  static constexpr size_t st_ph = st_src + ws_al16(4 * ST);
  static constexpr size_t st_red = st_ph + 8 * (size_t)ST;   // float [NB][NC][32]
  static constexpr size_t stage_bytes = ws_al16(st_red + (size_t)NB * NC * 32 * 4);
  static constexpr size_t off_stage = NWIN * win_bytes;
  static constexpr size_t off_bar = off_stage + D * stage_bytes;
  static constexpr size_t off_misc = off_bar + 8 * (3 * D + 2 * NWIN);
  static constexpr size_t off_soff = ws_al16(off_misc + 16);   // int64 [kSepOffCache]
  static constexpr size_t bytes = off_soff + 8 * (size_t)kSepOffCache;
  static constexpr size_t alloc = bytes + 1024;   // the layout starts at the first 1024-byte boundary
};

template <int S, int P, int G, int TILE, int ST, int D, int NWIN, int MINB>
__global__ void __launch_bounds__(WsDegridLayout<S, P, G, TILE, ST, D, NWIN>::NT, MINB)
    k_degrid_ws(const DegridArgs a, const int cls, const __grid_constant__ CUtensorMap gmap) {
  using L = WsDegridLayout<S, P, G, TILE, ST, D, NWIN>;
  constexpr int NC = L::NC, R = L::R, B = L::B, UB = L::UB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  int64_t* s_off = reinterpret_cast<int64_t*>(smem + L::off_soff);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* redy = full + D;
  uint64_t* empty = full + 2 * D;
  uint64_t* wfull = full + 3 * D;
  uint64_t* wempty = wfull + NWIN;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::off_misc);
  unsigned long long* err = a.err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const bool off_cached = a.n_sep_off <= kSepOffCache;
  if (off_cached)
    for (int i = tid; i < a.n_sep_off; i += L::NT) s_off[i] = a.sep_off[i];
  const int64_t* offs = off_cached ? s_off : a.sep_off;
  if (tid == 0) {
    for (int d = 0; d < D; ++d) {
      mbar_init(full + d, 32);
      mbar_init(redy + d, NC * 32);
      mbar_init(empty + d, 32);
    }
    for (int w = 0; w < NWIN; ++w) {
      mbar_init(wfull + w, 1);
      mbar_init(wempty + w, NC * 32);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------------------------------ producer
    if (lane == 0) prefetch_tensormap(&gmap);
    WsItemWalker walk;
    walk.init(a.class_range[cls], a.class_range[cls + 1], cls, TILE, ST, a.queue, a.items);
    const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
    auto load_ph = [&](const WsChunk& d, const SampleRec& rc) {
      return (a.phasor && d.valid && lane < d.nst) ? __ldg(a.phasor + rc.src) : make_float2(1.f, 0.f);
    };
    // loads run ahead of their use: the records three chunks, the phasors two
    WsChunk d0 = walk.next();
    WsChunk d1 = walk.next();
    WsChunk d2 = walk.next();
    SampleRec r0 = ws_load_rec(a.rec, d0, lane);
    SampleRec r1 = ws_load_rec(a.rec, d1, lane);
    SampleRec r2 = ws_load_rec(a.rec, d2, lane);
    float2 ph0 = load_ph(d0, r0);
    float2 ph1 = load_ph(d1, r1);
    int k = 0, ic = 0;
    unsigned tma_pending = 0;   // bit w: a window load whose completion nobody may have waited for
    int tma_use[NWIN];
#pragma unroll
    for (int w = 0; w < NWIN; ++w) tma_use[w] = 0;
    bool ok = true;
    while (d0.valid) {
      if (d0.flags & kWsFirst) {
        // the item's window: one TMA tile load into a free window
        const int w = ic % NWIN;
        if (!mbar_wait(wempty + w, ((ic / NWIN) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          fence_proxy_async_smem();
          unsigned char* dst = smem + (size_t)w * L::win_bytes;
          mbar_arrive_expect_tx(wfull + w, L::box_bytes);
          const int X0 = d0.xy & 0xffff, Y0 = d0.xy >> 16;
          if constexpr (P == 1) tma_load_2d(dst, &gmap, 2 * (X0 & ~1), Y0, wfull + w);
          else tma_load_3d(dst, &gmap, 0, X0, Y0, wfull + w);
        }
        tma_pending |= 1u << w;
        tma_use[w] = ic / NWIN;
        ++ic;
      }
      const int s = k % D;
      unsigned char* sg = smem + L::off_stage + (size_t)s * L::stage_bytes;
      if (!mbar_wait(empty + s, ((k / D) & 1) ^ 1, abort_flag, err)) {
        ok = false;
        break;
      }
      const int X0 = d0.xy & 0xffff, Y0 = d0.xy >> 16;
      const int pk = (r0.p0x - X0) | ((r0.p0y - Y0) << 8) | ((r0.p0x % S) << 16) | ((r0.p0y % S) << 24);
      const int nr = ws_runs(pk, d0.nst, lane, reinterpret_cast<int*>(sg + L::st_rs),
                             reinterpret_cast<int*>(sg + L::st_rpk));
      if (lane < d0.nst) {
        reinterpret_cast<int*>(sg + L::st_src)[lane] = a.rank > 1 ? r0.src * a.rank + r0.cf % a.rank : r0.src;
        reinterpret_cast<float2*>(sg + L::st_ph)[lane] = ph0;
        long long fxo, fyo;
        ws_rows<S>(offs, a.cf_shift, a.OS, r0, fxo, fyo);
        fence_proxy_async_smem();   // the consumers' reads of this stage come before the copies
        bulk_load(sg + L::st_fx + (size_t)lane * S * 8, sep2 + fxo, S * 8, full + s);
        bulk_load(sg + L::st_fy + (size_t)lane * 2 * S * 8, sep2 + fyo, S * 8, full + s);
        bulk_load(sg + L::st_fy + (size_t)lane * 2 * S * 8 + S * 8, sep2 + fyo, S * 8, full + s);
      }
      if (lane == 0) *reinterpret_cast<WsHeader*>(sg) = WsHeader{d0.nst, d0.flags, d0.xy, nr};
      if (!(a.withhold && k == 0)) {
        if (lane == 0) mbar_arrive_expect_tx(full + s, (unsigned)(d0.nst * 3 * S * 8));
        else mbar_arrive(full + s);
      }
      const WsChunk d3 = walk.next();
      const SampleRec r3 = ws_load_rec(a.rec, d3, lane);
      const float2 ph2 = load_ph(d2, r2);
      d0 = d1;
      d1 = d2;
      d2 = d3;
      r0 = r1;
      r1 = r2;
      r2 = r3;
      ph0 = ph1;
      ph1 = ph2;
      ++k;
    }
    if (ok && mbar_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
      if (lane == 0) *reinterpret_cast<WsHeader*>(smem + L::off_stage + (size_t)(k % D) * L::stage_bytes) =
          WsHeader{-1, 0, 0, 0};
      mbar_arrive(full + k % D);
    }
    if (!ok || *abort_flag) {
      // no consumer may wait for an issued window load any more: wait for it here (bounded)
      // before the CTA can exit
      volatile int never = 0;
#pragma unroll
      for (int w = 0; w < NWIN; ++w)
        if (tma_pending & (1u << w)) mbar_wait(wfull + w, tma_use[w] & 1, &never, err);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------------------ reduce warp
    for (int k = 0;; ++k) {
      unsigned char* sg = smem + L::off_stage + (size_t)(k % D) * L::stage_bytes;
      if (!mbar_wait(redy + k % D, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      if (h.nst < 0) break;
      const float* red = reinterpret_cast<const float*>(sg + L::st_red);
      const int* srcv = reinterpret_cast<const int*>(sg + L::st_src);
      const float2* phv = reinterpret_cast<const float2*>(sg + L::st_ph);
      const int nbat = (h.nst + B - 1) / B;
      const int comp = lane % (2 * P);
      for (int bi = 0; bi < nbat; ++bi) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < NC; ++w) v += red[(bi * NC + w) * 32 + lane];
        const float partner = __shfl_xor_sync(0xffffffffu, v, 1);
        const int j = bi * B + lane / (2 * P);
        if (j < h.nst) {
          const float2 ph = phv[j];
          const float out = (comp & 1) ? (v * ph.x - partner * ph.y) : (v * ph.x + partner * ph.y);
          float* o = a.vis_out + ((size_t)srcv[j] * a.vstride + a.voff) * 2 + comp;
          *o = a.accumulate == 0 ? out : a.accumulate > 0 ? *o + out : *o - out;
        }
      }
      mbar_arrive(empty + k % D);
    }
  } else {
    // ------------------------------------------------------------------------------ consumers
    const int ct = tid - 64, cw = ct >> 5;
    int rx, ry0;
    ws_owner<S, G>(ct, rx, ry0);
    float2 gc[R][P];
    int curY[R], Y[R];
    int curX = -1, tx = 0, rowoff = 0, prev_pk = -1, prev_row = -1;
    const float2* win = reinterpret_cast<const float2*>(smem);
    int ic = 0;
#pragma unroll
    for (int kk = 0; kk < R; ++kk) {
      curY[kk] = -1;
      Y[kk] = 0;
    }
    for (int k = 0;; ++k) {
      unsigned char* sg = smem + L::off_stage + (size_t)(k % D) * L::stage_bytes;
      if (!mbar_wait(full + k % D, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      if (h.nst < 0) {
        mbar_arrive(redy + k % D);   // the reduce warp learns of the end from this stage
        break;
      }
      if (h.flags & kWsFirst) {
        const int w = ic % NWIN;
        if (!mbar_wait(wfull + w, (ic / NWIN) & 1, abort_flag, err)) break;
        // P = 1: the box starts at the even pixel at or below X0 (see the layout)
        win = reinterpret_cast<const float2*>(smem + (size_t)w * L::win_bytes) + (P == 1 ? (h.xy & 1) : 0);
        curX = -1;
        prev_pk = -1;
        prev_row = -1;
#pragma unroll
        for (int kk = 0; kk < R; ++kk) curY[kk] = -1;
      }
      const int* rsv = reinterpret_cast<const int*>(sg + L::st_rs);
      const int* rpkv = reinterpret_cast<const int*>(sg + L::st_rpk);
      const float2* fyb = reinterpret_cast<const float2*>(sg + L::st_fy);
      const float2* fxb = reinterpret_cast<const float2*>(sg + L::st_fx);
      float* red = reinterpret_cast<float*>(sg + L::st_red);
      int r = 0, next_run = 0;   // the next run starts at sample next_run
      for (int j0 = 0; j0 < h.nst; j0 += B) {
        float vals[2 * P * B];
#pragma unroll
        for (int q = 0; q < 2 * P * B; ++q) vals[q] = 0.f;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int j = j0 + b;
          if (j < h.nst) {
            if (j == next_run) {
              const int pk = rpkv[r];
              ++r;
              next_run = r < h.nr ? rsv[r] : h.nst;
              if (pk != prev_pk) {
                prev_pk = pk;
                const int dx = pk & 0xff, mx = (pk >> 16) & 0xff;
                const int row = pk & 0xff00ff00;
                bool row_changed = false;
                if (row != prev_row) {
                  prev_row = row;
                  const int dy = (pk >> 8) & 0xff, my = (pk >> 24) & 0xff;
                  rowoff = S - my + ry0;
#pragma unroll
                  for (int kk = 0; kk < R; ++kk) {
                    int t = ry0 + kk * G - my;
                    t += (t < 0) ? S : 0;
                    Y[kk] = dy + t;
                  }
                  row_changed = true;
                }
                tx = rx - mx;
                tx += (tx < 0) ? S : 0;
                const int X = dx + tx;
                if (X != curX || row_changed) {
                  const bool xchg = X != curX;
#pragma unroll
                  for (int kk = 0; kk < R; ++kk) {
                    if (xchg || Y[kk] != curY[kk]) {
                      curY[kk] = Y[kk];
                      load_pols<P>(win + ((size_t)curY[kk] * UB + X) * P, gc[kk]);
                    }
                  }
                  curX = X;
                }
              }
            }
            const float2 fx = fxb[j * S + tx];
            const float2* fyp = fyb + j * 2 * S + rowoff;
            float2 part[P];
#pragma unroll
            for (int p = 0; p < P; ++p) part[p] = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
              const float2 f = fyp[kk * G];
#pragma unroll
              for (int p = 0; p < P; ++p) {
                part[p].x = fmaf(f.x, gc[kk][p].x, fmaf(-f.y, gc[kk][p].y, part[p].x));
                part[p].y = fmaf(f.x, gc[kk][p].y, fmaf(f.y, gc[kk][p].x, part[p].y));
              }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
              vals[b * 2 * P + 2 * p] = fx.x * part[p].x - fx.y * part[p].y;
              vals[b * 2 * P + 2 * p + 1] = fx.x * part[p].y + fx.y * part[p].x;
            }
          }
        }
        // reduce-scatter over the warp: lane l ends with component l of the batch
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
        red[((j0 / B) * NC + cw) * 32 + lane] = vals[0];
      }
      mbar_arrive(redy + k % D);
      if (h.flags & kWsLast) {
        mbar_arrive(wempty + ic % NWIN);
        ++ic;
      }
    }
  }
}

// ------------------------------------------------------------------------------ configurations

// Warp-specialised configuration per exact support (candidate 2 of cf_set_autotune): row groups of
// the gridding and degridding consumers, samples per stage, stages in the ring, windows, and CTAs
// per SM the launch bounds aim at.  The tile of first-tap positions per item is candidate 2's of
// kExactCand, for which the cp.async kernels are compiled too: they serve the calls these kernels
// cannot take (strided-pol element passes, which the TMA window cannot describe; misaligned
// buffers; grids above 32768 pixels).
struct WsCfg {
  int S, g_grid, g_degrid, st_grid, st_degrid, d_grid, d_degrid, nwin_grid, nwin_degrid, minb_grid, minb_degrid;
};
constexpr WsCfg kWsCfg[8] = {
    {8, 8, 8, 16, 16, 4, 4, 2, 2, 4, 4},
    {16, 8, 8, 16, 16, 4, 4, 2, 2, 2, 2},
    {24, 8, 8, 16, 16, 3, 3, 2, 2, 2, 2},
    {32, 8, 8, 16, 16, 3, 3, 1, 2, 2, 1},
    {40, 8, 8, 12, 16, 4, 3, 2, 2, 1, 1},
    {48, 8, 8, 8, 8, 3, 3, 1, 1, 1, 1},
    {56, 8, 8, 8, 8, 3, 3, 1, 1, 1, 1},
    {64, 8, 8, 4, 8, 3, 3, 1, 1, 1, 1},
};
constexpr WsCfg ws_cfg(int S) {
  for (const WsCfg& e : kWsCfg)
    if (e.S == S) return e;
  return WsCfg{S, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
}

template <int S, int P, int C = 2>
awg_status run_grid_ws(const GridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr WsCfg c = ws_cfg(S);
  constexpr int T = exact_cfg(S, C).tile;
  using L = WsGridLayout<S, P, c.g_grid, T, c.st_grid, c.d_grid, c.nwin_grid>;
  static_assert(L::alloc <= 227 * 1024, "gridding stages do not fit");
  auto kern = k_grid_ws<S, P, c.g_grid, T, c.st_grid, c.d_grid, c.nwin_grid, c.minb_grid>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::alloc));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, L::NT, L::alloc));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "warp-specialised gridding kernel does not fit on an SM");
  }
  kern<<<sms * bps, L::NT, L::alloc, st>>>(a, slot);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// The tensor map of the grid for the degridding windows (built by the caller, see launch.cu).
awg_status make_grid_tensor_map(CUtensorMap* map, const void* grid, int N, int P, int U, int UB, int rows);

template <int S, int P, int C = 2>
awg_status run_degrid_ws(const DegridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr WsCfg c = ws_cfg(S);
  constexpr int T = exact_cfg(S, C).tile;
  using L = WsDegridLayout<S, P, c.g_degrid, T, c.st_degrid, c.d_degrid, c.nwin_degrid>;
  static_assert(L::alloc <= 227 * 1024, "degridding stages do not fit");
  auto kern = k_degrid_ws<S, P, c.g_degrid, T, c.st_degrid, c.d_degrid, c.nwin_degrid, c.minb_degrid>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::alloc));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, L::NT, L::alloc));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "warp-specialised degridding kernel does not fit on an SM");
  }
  CUtensorMap map;
  awg_status s = make_grid_tensor_map(&map, a.grid, a.N, P, L::U, L::UB, L::U);
  if (s != AWG_OK) return s;
  kern<<<sms * bps, L::NT, L::alloc, st>>>(a, slot, map);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// Supports and pol counts of the warp-specialised kernels, in two halves (two translation units each).
#define AWG_FOR_WS_A(M) M(8, 1) M(8, 2) M(8, 4) M(16, 1) M(16, 2) M(16, 4) M(24, 1) M(24, 2) M(24, 4) M(32, 1) M(32, 2) M(32, 4)
#define AWG_FOR_WS_B(M) M(40, 1) M(40, 2) M(40, 4) M(48, 1) M(48, 2) M(48, 4) M(56, 1) M(56, 2) M(56, 4) M(64, 1) M(64, 2) M(64, 4)
// supports whose candidate-3 windows are wider than 64 (degridding on the warp-specialised kernel)
#define AWG_FOR_WS3(M) M(64, 1) M(64, 2) M(64, 4)
#define AWG_DECLARE_GRID_WS(S, P) extern template awg_status run_grid_ws<S, P, 2>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_WS(S, P) \
  extern template awg_status run_degrid_ws<S, P, 2>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_WS3(S, P) \
  extern template awg_status run_degrid_ws<S, P, 3>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_WS(S, P) template awg_status run_grid_ws<S, P, 2>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_WS(S, P) \
  template awg_status run_degrid_ws<S, P, 2>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_WS3(S, P) \
  template awg_status run_degrid_ws<S, P, 3>(const DegridArgs&, int, int, cudaStream_t);

}  // namespace awg
