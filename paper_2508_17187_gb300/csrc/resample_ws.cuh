// Warp-specialised gridding and degridding with separable rank-1 CF records on the exact
// supports (the W-projection schedule): the arithmetic of resample_sep.cuh, with the per-chunk
// CTA barriers replaced by a ring of shared-memory stages handed over on mbarriers.
//
// Roles (one persistent CTA pulls work items of one support from its queue):
//  * warp 0, the producer, walks the CTA's items chunk by chunk.  For chunk k it copies the records
//    of chunk k + 1 and the factor rows, visibilities, weights and phasors of chunk k with cp.async,
//    and while those are in flight it finishes chunk k - 1 (gridding: the table
//    alpha[j][rx][p] = conj(fx_j[(rx - mx_j) mod S]) w_jp V_jp, the weight sums) and hands its
//    stage to the consumers.  fy is stored rotated, fyr[j][ry] = fy_j[(ry - my_j) mod S], so a
//    consumer finds the factor of each of its rows at a fixed offset.
//  * the consumer warps own the taps by residue as in resample_sep.cuh (thread: column residue rx,
//    rows ry0 + k G) and run only the multiply-add loop over the samples of each stage; a stage is
//    released to the producer when every consumer thread has read it.
//  * gridding: warp 1 flushes.  The consumers accumulate an item in one of NWIN shared windows and
//    hand it to the flush warp, which adds it to the grid (one vector atomic per non-zero pixel)
//    and zeroes it, while the consumers go on with the next item in the other window.
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
  int pad;
};

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

// ------------------------------------------------------------------------------------ gridding

template <int S, int P, int G, int TILE, int ST, int D, int NWIN>
struct WsGridLayout {
  static_assert(S % G == 0 && (S * G) % 32 == 0, "row groups must divide S and fill whole warps");
  static constexpr int NC = S * G / 32;          // consumer warps
  static constexpr int NT = 32 * (NC + 2);       // + producer + flush warp
  static constexpr int R = S / G;                // rows per consumer thread
  static constexpr int U = TILE + S - 1;
  static constexpr int UU = U * U;
  static constexpr size_t win_bytes = ws_al16((size_t)UU * P * 8);   // pol-planar float2 [P][U][U]
  // a stage: header, packed positions, rotated fy rows, the alpha table
  static constexpr size_t st_pk = 16;
  static constexpr size_t st_fy = st_pk + ws_al16(4 * ST);
  static constexpr size_t st_al = st_fy + (size_t)ST * S * 8;
  static constexpr size_t stage_bytes = ws_al16(st_al + (size_t)ST * S * P * 8);
  // a producer staging slot: records, fx rows, visibilities, weights, phasors, derived data
  static constexpr size_t ps_rec = 0;
  static constexpr size_t ps_fx = ps_rec + 16 * (size_t)ST;
  static constexpr size_t ps_v = ps_fx + (size_t)ST * S * 8;
  static constexpr size_t ps_w = ps_v + (size_t)ST * P * 8;
  static constexpr size_t ps_ph = ps_w + ws_al16(4 * (size_t)ST * P);
  static constexpr size_t ps_off = ps_ph + 8 * (size_t)ST;   // long long [ST][2]: fx, fy row offsets
  static constexpr size_t ps_src = ps_off + 16 * (size_t)ST; // int [ST]
  static constexpr size_t ps_pk = ps_src + ws_al16(4 * (size_t)ST);
  static constexpr size_t ps_wt0 = ps_pk + ws_al16(4 * (size_t)ST);   // int [ST]: adds its weight
  static constexpr size_t pstage_bytes = ws_al16(ps_wt0 + 4 * (size_t)ST);
  static constexpr size_t off_stage = NWIN * win_bytes;
  static constexpr size_t off_pstage = off_stage + D * stage_bytes;
  static constexpr size_t off_bar = off_pstage + 2 * pstage_bytes;
  static constexpr size_t off_misc = off_bar + 8 * (2 * D + 2 * NWIN);
  static constexpr size_t off_soff = ws_al16(off_misc + 16 + 4 * NWIN);   // int64 [kSepOffCache]
  static constexpr size_t bytes = off_soff + 8 * (size_t)kSepOffCache;
  static constexpr size_t alloc = bytes + 1024;   // the layout starts at the first 1024-byte boundary
};

// The producer's walk over the CTA's items: descriptor of one chunk.
struct WsChunk {
  int start, nst, xy, flags;
  bool valid;
};

struct WsItemWalker {
  int begin, end, cls, tile;
  int32_t* queue;
  const WorkItem* items;
  int st;          // samples per chunk
  int it;          // current item (>= end: none)
  WorkItem wi;
  int c, nch;      // next chunk of the current item, chunks of the item
  int pending;     // index of the item after the current one (fetched when the current one starts)

  __device__ __forceinline__ int fetch() {
    int v = 0;
    if ((threadIdx.x & 31) == 0) v = begin + atomicAdd(queue + cls, 1);
    return __shfl_sync(0xffffffffu, v, 0);
  }
  __device__ __forceinline__ void load(int i) {
    it = i;
    if (it < end) {
      wi = items[it];
      nch = (wi.count + st - 1) / st;
      c = 0;
      pending = fetch();
    }
  }
  __device__ __forceinline__ void init() { load(fetch()); }
  __device__ __forceinline__ WsChunk next() {
    WsChunk d{0, 0, 0, 0, false};
    if (it < end && c >= nch) load(pending);
    if (it >= end) return d;
    d.start = wi.start + c * st;
    d.nst = min(st, wi.count - c * st);
    d.xy = (wi.tile_x * tile) | ((wi.tile_y * tile) << 16);
    d.flags = (c == 0 ? kWsFirst : 0) | (c == nch - 1 ? kWsLast : 0);
    d.valid = true;
    ++c;
    return d;
  }
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
  uint64_t* wfull = full + 2 * D;
  uint64_t* wempty = wfull + NWIN;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::off_misc);
  int* win_info = reinterpret_cast<int*>(smem + L::off_misc + 16);
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
    for (int w = 0; w < NWIN; ++w) {
      mbar_init(wfull + w, NC * 32);
      mbar_init(wempty + w, 32);
    }
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
    WsItemWalker walk{a.class_range[cls], a.class_range[cls + 1], cls, TILE, a.queue, a.items, ST, 0, {}, 0, 0, 0};
    walk.init();
    const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
    auto pst = [&](int i) { return smem + L::off_pstage + (size_t)(i & 1) * L::pstage_bytes; };
    auto stg = [&](int i) { return smem + L::off_stage + (size_t)(i % D) * L::stage_bytes; };
    auto issue_recs = [&](const WsChunk& d, unsigned char* ps) {
      if (lane < d.nst) cp_async(ps + L::ps_rec + 16 * lane, a.rec + d.start + lane, 16);
    };
    WsChunk dk = walk.next();
    if (dk.valid) issue_recs(dk, pst(0));
    cp_async_commit();
    WsChunk dprev{0, 0, 0, 0, false};
    int k = 0;
    bool ok = true;
    for (;;) {
      cp_async_wait_all();
      __syncwarp();
      const WsChunk dn = dk.valid ? walk.next() : WsChunk{0, 0, 0, 0, false};
      if (dk.valid) {
        unsigned char* ps = pst(k);
        unsigned char* sg = stg(k);
        if (!mbar_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
          ok = false;
          break;
        }
        // derive chunk k from its records: packed window position, factor-row offsets, source row
        if (lane < dk.nst) {
          const SampleRec rc = reinterpret_cast<const SampleRec*>(ps + L::ps_rec)[lane];
          const int X0 = dk.xy & 0xffff, Y0 = dk.xy >> 16;
          const int mx = rc.p0x % S, my = rc.p0y % S;
          const int pk = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | (mx << 16) | (my << 24);
          const long long base = offs[a.cf_shift + rc.cf];
          reinterpret_cast<long long*>(ps + L::ps_off)[2 * lane] = base + (long long)rc.ox * S;
          reinterpret_cast<long long*>(ps + L::ps_off)[2 * lane + 1] =
              base + (long long)(a.OS + 1) * S + (long long)rc.oy * S;
          reinterpret_cast<int*>(ps + L::ps_src)[lane] = rc.src;
          reinterpret_cast<int*>(ps + L::ps_pk)[lane] = pk;
          reinterpret_cast<int*>(ps + L::ps_wt0)[lane] = (a.rank == 1 || rc.cf % a.rank == 0) ? 1 : 0;
          reinterpret_cast<int*>(sg + L::st_pk)[lane] = pk;
        }
        __syncwarp();
        // fy rotated into the stage, fx as stored into the staging slot (8-byte copies)
        const long long* off = reinterpret_cast<const long long*>(ps + L::ps_off);
        const int* pkv = reinterpret_cast<const int*>(ps + L::ps_pk);
        float2* fyr = reinterpret_cast<float2*>(sg + L::st_fy);
        float2* fxs = reinterpret_cast<float2*>(ps + L::ps_fx);
        for (int i = lane; i < dk.nst * S; i += 32) {
          const int j = i / S, t = i - j * S;
          int ry = t + ((pkv[j] >> 24) & 0xff);   // fyr[j][(t + my) mod S] = fy_j[t]
          ry -= (ry >= S) ? S : 0;
          cp_async(fyr + j * S + ry, sep2 + off[2 * j + 1] + t, 8);
          cp_async(fxs + i, sep2 + off[2 * j] + t, 8);
        }
        if (lane < dk.nst) {
          const size_t s = (size_t)reinterpret_cast<const int*>(ps + L::ps_src)[lane];
          const float* vp = a.vis + s * P * 2;
          const float* wp = a.weight + s * P;
          float2* v = reinterpret_cast<float2*>(ps + L::ps_v) + lane * P;
          float* w = reinterpret_cast<float*>(ps + L::ps_w) + lane * P;
          if constexpr (P == 4) {
            cp_async(v, vp, 16);
            cp_async(v + 2, vp + 4, 16);
            cp_async(w, wp, 16);
          } else if constexpr (P == 2) {
            cp_async(v, vp, 16);
            cp_async(w, wp, 8);
          } else {
            cp_async(v, vp, 8);
            cp_async(w, wp, 4);
          }
          float2* ph = reinterpret_cast<float2*>(ps + L::ps_ph) + lane;
          if (a.phasor) {
            const SampleRec rc = reinterpret_cast<const SampleRec*>(ps + L::ps_rec)[lane];
            cp_async(ph, a.phasor + rc.src, 8);
          } else {
            *ph = make_float2(1.f, 0.f);
          }
        }
        if (dn.valid) issue_recs(dn, pst(k + 1));
        cp_async_commit();
      }
      if (dprev.valid) {
        // finish chunk k - 1 (its copies landed at the top of this pass): alpha, weights, header
        unsigned char* ps = pst(k - 1);
        unsigned char* sg = stg(k - 1);
        const int nst = dprev.nst;
        const float2* v = reinterpret_cast<const float2*>(ps + L::ps_v);
        const float* w = reinterpret_cast<const float*>(ps + L::ps_w);
        const float2* ph = reinterpret_cast<const float2*>(ps + L::ps_ph);
        if (lane < nst && reinterpret_cast<const int*>(ps + L::ps_wt0)[lane]) {
#pragma unroll
          for (int p = 0; p < P; ++p) wsum[p] += (double)w[lane * P + p];
        }
        const int* pkv = reinterpret_cast<const int*>(ps + L::ps_pk);
        const float2* fxs = reinterpret_cast<const float2*>(ps + L::ps_fx);
        float2* al = reinterpret_cast<float2*>(sg + L::st_al);
        for (int i = lane; i < nst * S; i += 32) {
          const int j = i / S, rx = i - j * S;
          int tx = rx - ((pkv[j] >> 16) & 0xff);
          tx += (tx < 0) ? S : 0;
          const float2 f = fxs[j * S + tx];
          const float2 phj = ph[j];
          float2 o[P];
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const float wv = w[j * P + p];
            const float2 vv = v[j * P + p];
            const float xr = wv * vv.x, xi = wv * vv.y;
            const float ar = xr * phj.x - xi * phj.y, ai = xr * phj.y + xi * phj.x;
            o[p] = make_float2(f.x * ar + f.y * ai, f.x * ai - f.y * ar);   // conj(fx) w V ph
          }
          float2* dst = al + (size_t)i * P;
          if constexpr (P % 2 == 0) {
#pragma unroll
            for (int q = 0; q < P / 2; ++q)
              reinterpret_cast<float4*>(dst)[q] = make_float4(o[2 * q].x, o[2 * q].y, o[2 * q + 1].x, o[2 * q + 1].y);
          } else {
            dst[0] = o[0];
          }
        }
        if (lane == 0) *reinterpret_cast<WsHeader*>(sg) = WsHeader{nst, dprev.flags, dprev.xy, 0};
        if (!(a.withhold && k == 1)) mbar_arrive(full + (k - 1) % D);
      }
      if (!dk.valid) break;
      dprev = dk;
      dk = dn;
      ++k;
    }
    if (ok && mbar_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
      if (lane == 0) *reinterpret_cast<WsHeader*>(stg(k)) = WsHeader{-1, 0, 0, 0};
      mbar_arrive(full + k % D);
    }
    cp_async_wait_all();
#pragma unroll
    for (int p = 0; p < P; ++p) {
      double s = wsum[p];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0 && s != 0.0 && a.sumwt) atomicAdd(a.sumwt + p, s);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------------------ flush warp
    for (int ic = 0;; ++ic) {
      const int w = ic % NWIN;
      if (!mbar_wait(wfull + w, (ic / NWIN) & 1, abort_flag, err)) break;
      const int info = win_info[w];
      if (info < 0) break;
      const int X0 = info & 0xffff, Y0 = info >> 16;
      float2* win = reinterpret_cast<float2*>(smem + (size_t)w * L::win_bytes);
      for (int i = lane; i < UU; i += 32) {
        const int ly = i / U, lx = i - ly * U;
        const int gy = Y0 + ly, gx = X0 + lx;
        float2 v[P];
        bool nz = false;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          v[p] = win[p * UU + i];
          nz |= (v[p].x != 0.f) || (v[p].y != 0.f);
        }
        if (nz) {
#pragma unroll
          for (int p = 0; p < P; ++p) win[p * UU + i] = make_float2(0.f, 0.f);
          if (gy < a.N && gx < a.N) flush_pixel<P>(a, ((size_t)gy * a.N + gx) * P, v);
        }
      }
      mbar_arrive(wempty + w);
    }
  } else {
    // ------------------------------------------------------------------------------ consumers
    const int ct = tid - 64;
    int rx, ry0;
    ws_owner<S, G>(ct, rx, ry0);
    float2 acc[R][P];
    int curY[R], Y[R];
    int curX = -1, prev_pk = -1, prev_row = -1;
    float2* win = reinterpret_cast<float2*>(smem);
    int ic = 0;
    for (int k = 0;; ++k) {
      unsigned char* sg = smem + L::off_stage + (size_t)(k % D) * L::stage_bytes;
      if (!mbar_wait(full + k % D, (k / D) & 1, abort_flag, err)) break;
      const WsHeader h = *reinterpret_cast<const WsHeader*>(sg);
      const int w = ic % NWIN;
      if (h.nst < 0 || (h.flags & kWsFirst)) {
        // a new item (or the end): its window must have been flushed
        if (!mbar_wait(wempty + w, ((ic / NWIN) & 1) ^ 1, abort_flag, err)) break;
        if (ct == 0) win_info[w] = h.nst < 0 ? -1 : h.xy;
        if (h.nst < 0) {
          mbar_arrive(wfull + w);
          break;
        }
        win = reinterpret_cast<float2*>(smem + (size_t)w * L::win_bytes);
        curX = -1;
        prev_pk = -1;
        prev_row = -1;
#pragma unroll
        for (int kk = 0; kk < R; ++kk) {
          curY[kk] = -1;
          Y[kk] = 0;
#pragma unroll
          for (int p = 0; p < P; ++p) acc[kk][p] = make_float2(0.f, 0.f);
        }
      }
      const int* pkv = reinterpret_cast<const int*>(sg + L::st_pk);
      const float2* fyb = reinterpret_cast<const float2*>(sg + L::st_fy) + ry0;
      const float2* alb = reinterpret_cast<const float2*>(sg + L::st_al) + rx * P;
      for (int j = 0; j < h.nst; ++j) {
        const int pk = pkv[j];
        float2 al[P];
        load_pols<P>(alb + j * S * P, al);
        float2 f[R];
#pragma unroll
        for (int kk = 0; kk < R; ++kk) f[kk] = fyb[j * S + kk * G];
        if (pk != prev_pk) {   // the first tap moved (the same test in every consumer thread)
          prev_pk = pk;
          const int dx = pk & 0xff, mx = (pk >> 16) & 0xff;
          const int row = pk & 0xff00ff00;
          bool row_changed = false;
          if (row != prev_row) {
            prev_row = row;
            const int dy = (pk >> 8) & 0xff, my = (pk >> 24) & 0xff;
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
              int t = ry0 + kk * G - my;
              t += (t < 0) ? S : 0;
              Y[kk] = dy + t;
            }
            row_changed = true;
          }
          int tx = rx - mx;
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
#pragma unroll
        for (int kk = 0; kk < R; ++kk) {
#pragma unroll
          for (int p = 0; p < P; ++p) {   // acc += conj(fy) alpha
            acc[kk][p].x = fmaf(f[kk].x, al[p].x, fmaf(f[kk].y, al[p].y, acc[kk][p].x));
            acc[kk][p].y = fmaf(f[kk].x, al[p].y, fmaf(-f[kk].y, al[p].x, acc[kk][p].y));
          }
        }
      }
      mbar_arrive(empty + k % D);
      if (h.flags & kWsLast) {
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
        mbar_arrive(wfull + w);
        ++ic;
      }
    }
  }
}

// ---------------------------------------------------------------------------------- degridding

template <int S, int P, int G, int TILE, int ST, int D, int NWIN>
struct WsDegridLayout {
  static_assert(S % G == 0 && (S * G) % 32 == 0, "row groups must divide S and fill whole warps");
  static constexpr int NC = S * G / 32;
  static constexpr int NT = 32 * (NC + 2);        // + producer + reduce warp
  static constexpr int R = S / G;
  static constexpr int U = TILE + S - 1;
  static constexpr int B = 32 / (2 * P);          // samples per butterfly batch
  static constexpr int NB = (ST + B - 1) / B;     // batches per stage
  // window as the TMA tile lands: P >= 2: [U][U][P] c64 (3-D box (2P, U, U)); P = 1: rows of UB
  // pixels, UB = U rounded up to even (2-D box (2 UB, U): a whole number of 16-byte units per row)
  static constexpr int UB = (P == 1) ? ((U + 1) & ~1) : U;
  static constexpr unsigned box_bytes = (unsigned)U * UB * P * 8;
  static constexpr size_t win_bytes = ws_al1k(box_bytes);
  static constexpr size_t st_pk = 16;
  static constexpr size_t st_fy = st_pk + ws_al16(4 * ST);
  static constexpr size_t st_fx = st_fy + (size_t)ST * S * 8;
  static constexpr size_t st_src = st_fx + (size_t)ST * S * 8;
  static constexpr size_t st_ph = st_src + ws_al16(4 * ST);
  static constexpr size_t st_red = st_ph + 8 * (size_t)ST;   // float [NB][NC][32]
  static constexpr size_t stage_bytes = ws_al16(st_red + (size_t)NB * NC * 32 * 4);
  static constexpr size_t off_stage = NWIN * win_bytes;
  static constexpr size_t off_rec = off_stage + D * stage_bytes;   // SampleRec [2][ST]
  static constexpr size_t off_drv = off_rec + 2 * 16 * (size_t)ST;  // long long [ST][2], int mx|my [ST]
  static constexpr size_t off_bar = off_drv + ws_al16(16 * (size_t)ST + 4 * (size_t)ST);
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
    WsItemWalker walk{a.class_range[cls], a.class_range[cls + 1], cls, TILE, a.queue, a.items, ST, 0, {}, 0, 0, 0};
    walk.init();
    const float2* sep2 = reinterpret_cast<const float2*>(a.sep);
    auto recs = [&](int i) { return reinterpret_cast<SampleRec*>(smem + L::off_rec) + (i & 1) * ST; };
    auto stg = [&](int i) { return smem + L::off_stage + (size_t)(i % D) * L::stage_bytes; };
    long long* drv_off = reinterpret_cast<long long*>(smem + L::off_drv);
    int* drv_m = reinterpret_cast<int*>(smem + L::off_drv + 16 * (size_t)ST);
    WsChunk dk = walk.next();
    if (dk.valid && lane < dk.nst) cp_async(recs(0) + lane, a.rec + dk.start + lane, 16);
    cp_async_commit();
    WsChunk dprev{0, 0, 0, 0, false};
    int k = 0, ic = 0;
    unsigned tma_pending = 0;   // bit w: a window load whose completion nobody may have waited for
    int tma_use[NWIN];
#pragma unroll
    for (int w = 0; w < NWIN; ++w) tma_use[w] = 0;
    bool ok = true;
    for (;;) {
      cp_async_wait_all();
      __syncwarp();
      // chunk k - 1 has landed: hand it over first, so that the consumers can finish its item
      // while this warp waits below for a free window or stage
      if (dprev.valid) {
        if (lane == 0) *reinterpret_cast<WsHeader*>(stg(k - 1)) = WsHeader{dprev.nst, dprev.flags, dprev.xy, 0};
        if (!(a.withhold && k == 1)) mbar_arrive(full + (k - 1) % D);
      }
      if (!dk.valid) break;
      const WsChunk dn = walk.next();
      if (dk.flags & kWsFirst) {
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
          const int X0 = dk.xy & 0xffff, Y0 = dk.xy >> 16;
          if constexpr (P == 1) tma_load_2d(dst, &gmap, 2 * X0, Y0, wfull + w);
          else tma_load_3d(dst, &gmap, 0, X0, Y0, wfull + w);
        }
        tma_pending |= 1u << w;
        tma_use[w] = ic / NWIN;
        ++ic;
      }
      unsigned char* sg = stg(k);
      if (!mbar_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
        ok = false;
        break;
      }
      const SampleRec* rv = recs(k);
      if (lane < dk.nst) {
        const SampleRec rc = rv[lane];
        const int X0 = dk.xy & 0xffff, Y0 = dk.xy >> 16;
        const int mx = rc.p0x % S, my = rc.p0y % S;
        const long long base = offs[a.cf_shift + rc.cf];
        drv_off[2 * lane] = base + (long long)rc.ox * S;
        drv_off[2 * lane + 1] = base + (long long)(a.OS + 1) * S + (long long)rc.oy * S;
        drv_m[lane] = mx | (my << 8);
        reinterpret_cast<int*>(sg + L::st_pk)[lane] = (rc.p0x - X0) | ((rc.p0y - Y0) << 8) | (mx << 16) | (my << 24);
        reinterpret_cast<int*>(sg + L::st_src)[lane] = a.rank > 1 ? rc.src * a.rank + rc.cf % a.rank : rc.src;
        float2* ph = reinterpret_cast<float2*>(sg + L::st_ph) + lane;
        if (a.phasor) cp_async(ph, a.phasor + rc.src, 8);
        else *ph = make_float2(1.f, 0.f);
      }
      __syncwarp();
      float2* fyr = reinterpret_cast<float2*>(sg + L::st_fy);
      float2* fxr = reinterpret_cast<float2*>(sg + L::st_fx);
      for (int i = lane; i < dk.nst * S; i += 32) {
        const int j = i / S, t = i - j * S;
        const int m = drv_m[j];
        int ry = t + (m >> 8);        // fyr[j][(t + my) mod S] = fy_j[t]
        ry -= (ry >= S) ? S : 0;
        int rx = t + (m & 0xff);      // fxr[j][(t + mx) mod S] = fx_j[t]
        rx -= (rx >= S) ? S : 0;
        cp_async(fyr + j * S + ry, sep2 + drv_off[2 * j + 1] + t, 8);
        cp_async(fxr + j * S + rx, sep2 + drv_off[2 * j] + t, 8);
      }
      if (dn.valid && lane < dn.nst) cp_async(recs(k + 1) + lane, a.rec + dn.start + lane, 16);
      cp_async_commit();
      __syncwarp();   // every lane has read drv_* before the next pass rewrites them
      dprev = dk;
      dk = dn;
      ++k;
    }
    if (ok && mbar_wait(empty + k % D, ((k / D) & 1) ^ 1, abort_flag, err)) {
      if (lane == 0) *reinterpret_cast<WsHeader*>(stg(k)) = WsHeader{-1, 0, 0, 0};
      mbar_arrive(full + k % D);
    }
    cp_async_wait_all();
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
          *o = a.accumulate ? *o + out : out;
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
    int curX = -1, prev_pk = -1, prev_row = -1;
    const float2* win = reinterpret_cast<const float2*>(smem);
    int ic = 0;
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
        win = reinterpret_cast<const float2*>(smem + (size_t)w * L::win_bytes);
        curX = -1;
        prev_pk = -1;
        prev_row = -1;
#pragma unroll
        for (int kk = 0; kk < R; ++kk) {
          curY[kk] = -1;
          Y[kk] = 0;
        }
      }
      const int* pkv = reinterpret_cast<const int*>(sg + L::st_pk);
      const float2* fyb = reinterpret_cast<const float2*>(sg + L::st_fy) + ry0;
      const float2* fxb = reinterpret_cast<const float2*>(sg + L::st_fx) + rx;
      float* red = reinterpret_cast<float*>(sg + L::st_red);
      for (int j0 = 0; j0 < h.nst; j0 += B) {
        float vals[2 * P * B];
#pragma unroll
        for (int q = 0; q < 2 * P * B; ++q) vals[q] = 0.f;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int j = j0 + b;
          if (j < h.nst) {
            const int pk = pkv[j];
            const float2 fx = fxb[j * S];
            float2 f[R];
#pragma unroll
            for (int kk = 0; kk < R; ++kk) f[kk] = fyb[j * S + kk * G];
            if (pk != prev_pk) {
              prev_pk = pk;
              const int dx = pk & 0xff, mx = (pk >> 16) & 0xff;
              const int row = pk & 0xff00ff00;
              bool row_changed = false;
              if (row != prev_row) {
                prev_row = row;
                const int dy = (pk >> 8) & 0xff, my = (pk >> 24) & 0xff;
#pragma unroll
                for (int kk = 0; kk < R; ++kk) {
                  int t = ry0 + kk * G - my;
                  t += (t < 0) ? S : 0;
                  Y[kk] = dy + t;
                }
                row_changed = true;
              }
              int tx = rx - mx;
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
            float2 part[P];
#pragma unroll
            for (int p = 0; p < P; ++p) part[p] = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < R; ++kk) {
#pragma unroll
              for (int p = 0; p < P; ++p) {
                part[p].x = fmaf(f[kk].x, gc[kk][p].x, fmaf(-f[kk].y, gc[kk][p].y, part[p].x));
                part[p].y = fmaf(f[kk].x, gc[kk][p].y, fmaf(f[kk].y, gc[kk][p].x, part[p].y));
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
  int S, g_grid, g_degrid, st_grid, st_degrid, d, nwin_grid, nwin_degrid, minb_grid, minb_degrid;
};
constexpr WsCfg kWsCfg[8] = {
    {8, 8, 8, 16, 16, 4, 2, 2, 4, 4},
    {16, 8, 8, 16, 16, 4, 2, 2, 2, 2},
    {24, 8, 8, 16, 16, 3, 1, 2, 2, 2},
    {32, 8, 8, 16, 16, 3, 1, 2, 2, 1},
    {40, 8, 8, 12, 16, 3, 2, 2, 1, 1},
    {48, 8, 8, 8, 8, 3, 1, 2, 1, 1},
    {56, 8, 8, 8, 8, 3, 1, 1, 1, 1},
    {64, 8, 8, 4, 8, 3, 1, 1, 1, 1},
};
constexpr WsCfg ws_cfg(int S) {
  for (const WsCfg& e : kWsCfg)
    if (e.S == S) return e;
  return WsCfg{S, 0, 0, 0, 0, 0, 0, 0, 0, 0};
}

template <int S, int P>
awg_status run_grid_ws(const GridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr WsCfg c = ws_cfg(S);
  constexpr int T = exact_cfg(S, 2).tile;
  using L = WsGridLayout<S, P, c.g_grid, T, c.st_grid, c.d, c.nwin_grid>;
  static_assert(L::alloc <= 227 * 1024, "gridding stages do not fit");
  auto kern = k_grid_ws<S, P, c.g_grid, T, c.st_grid, c.d, c.nwin_grid, c.minb_grid>;
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
awg_status make_grid_tensor_map(CUtensorMap* map, const void* grid, int N, int P, int U, int UB);

template <int S, int P>
awg_status run_degrid_ws(const DegridArgs& a, int slot, int sms, cudaStream_t st) {
  constexpr WsCfg c = ws_cfg(S);
  constexpr int T = exact_cfg(S, 2).tile;
  using L = WsDegridLayout<S, P, c.g_degrid, T, c.st_degrid, c.d, c.nwin_degrid>;
  static_assert(L::alloc <= 227 * 1024, "degridding stages do not fit");
  auto kern = k_degrid_ws<S, P, c.g_degrid, T, c.st_degrid, c.d, c.nwin_degrid, c.minb_degrid>;
  static int bps = 0;
  if (bps == 0) {
    AWG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::alloc));
    AWG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, L::NT, L::alloc));
    if (bps < 1) return set_error(AWG_ERR_CUDA, "warp-specialised degridding kernel does not fit on an SM");
  }
  CUtensorMap map;
  awg_status s = make_grid_tensor_map(&map, a.grid, a.N, P, L::U, L::UB);
  if (s != AWG_OK) return s;
  kern<<<sms * bps, L::NT, L::alloc, st>>>(a, slot, map);
  AWG_CUDA_TRY(cudaGetLastError());
  count_launches(1);
  return AWG_OK;
}

// Supports and pol counts of the warp-specialised kernels, in two halves (two translation units each).
#define AWG_FOR_WS_A(M) M(8, 1) M(8, 2) M(8, 4) M(16, 1) M(16, 2) M(16, 4) M(24, 1) M(24, 2) M(24, 4) M(32, 1) M(32, 2) M(32, 4)
#define AWG_FOR_WS_B(M) M(40, 1) M(40, 2) M(40, 4) M(48, 1) M(48, 2) M(48, 4) M(56, 1) M(56, 2) M(56, 4) M(64, 1) M(64, 2) M(64, 4)
#define AWG_DECLARE_GRID_WS(S, P) extern template awg_status run_grid_ws<S, P>(const GridArgs&, int, int, cudaStream_t);
#define AWG_DECLARE_DEGRID_WS(S, P) \
  extern template awg_status run_degrid_ws<S, P>(const DegridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_GRID_WS(S, P) template awg_status run_grid_ws<S, P>(const GridArgs&, int, int, cudaStream_t);
#define AWG_INSTANTIATE_DEGRID_WS(S, P) \
  template awg_status run_degrid_ws<S, P>(const DegridArgs&, int, int, cudaStream_t);

}  // namespace awg
