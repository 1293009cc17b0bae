// Internal declarations of the awgrid library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "awgrid.h"

namespace awg {

// NVTX range over one host call of the library (a profiler shows the call's extent on the CPU
// timeline next to the kernels it launches; without a profiler attached the calls cost nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr double kCLight = 299792458.0;
constexpr int kMaxSupport = 64;
constexpr int kNumClasses = 6;
constexpr int kItemChunk = 1024;  // samples per work item at most (bounds the queue tail)

// Kernel classes: supports in (smax of the previous class, smax] run in one template instance
// with nt threads per CTA and tile x tile sample-start positions per work item.
struct ClassCfg {
  int smax, nt, tile;
};
constexpr ClassCfg kClasses[kNumClasses] = {
    {8, 64, 32}, {16, 128, 32}, {24, 192, 32}, {32, 256, 32}, {48, 256, 16}, {64, 256, 8}};

// Class of a support (the smax column of kClasses, spelled out so device code can call it).
__host__ __device__ constexpr int class_of_support(int S) {
  return S <= 8 ? 0 : S <= 16 ? 1 : S <= 24 ? 2 : S <= 32 ? 3 : S <= 48 ? 4 : S <= 64 ? 5 : -1;
}

// Separable kernels specialised for one support S (the W-projection schedule's multiples of 8):
// row groups G of the gridding and degridding kernels (each thread owns S / G rows of one column
// residue; S * G threads per CTA, a whole number of warps), the tile of first-tap positions per
// work item, which the plan uses for these supports when the CF set is separable, and the
// samples staged per chunk.  Small tiles let two CTAs share an SM; deeper stages spread the
// barriers of a chunk (and the unequal flush work between warps) over more samples, which won
// where two CTAs still fit (candidate 1 of supports 24-56: 1-3% on the W-projection workload).
// Every support has kNumCand compiled candidates; candidate 0 is the default and cf_set_autotune
// picks per support by timing.  Candidate 2 is the warp-specialised pair of kernels, candidate 3
// the tensor-core pair (the warp-specialised degridding kernel where a window is wider than 64).
// Fused multi-term kernels take the tiles of candidates 0 and 1.  The supports listed here and
// AWG_FOR_EXACT_AND_POLS must agree.
struct ExactCfg {
  int S, g_grid, g_degrid, tile, stage;
};
constexpr int kNumCand = 4;
constexpr ExactCfg kExactCand[kNumCand][8] = {
    {
        {8, 8, 8, 32, 16},
        {16, 8, 8, 16, 8},
        {24, 8, 8, 16, 8},
        {32, 8, 8, 16, 8},
        {40, 8, 8, 8, 8},
        {48, 16, 8, 16, 16},
        {56, 8, 8, 16, 8},
        {64, 8, 8, 8, 8},
    },
    {
        {8, 8, 8, 16, 8},
        {16, 16, 16, 32, 16},
        {24, 8, 8, 8, 16},
        {32, 8, 8, 8, 16},
        {40, 8, 8, 8, 12},
        {48, 8, 8, 8, 16},
        {56, 8, 8, 8, 16},
        {64, 8, 8, 8, 4},
    },
    {
        // candidate 2: the warp-specialised kernels (resample_ws.cuh) with these tiles; the
        // cp.async kernels compiled with the same tiles serve the calls those cannot take
        {8, 8, 8, 16, 8},
        {16, 8, 8, 16, 8},
        {24, 8, 8, 8, 16},
        {32, 8, 8, 8, 16},
        {40, 8, 8, 8, 12},
        {48, 8, 8, 8, 16},
        {56, 8, 8, 8, 16},
        {64, 8, 8, 8, 4},
    },
    {
        // candidate 3: the tensor-core kernels (resample_mma.cuh, resample_mma_dg.cuh) with these
        // tiles (window side S + tile - 1 at or just below a multiple of 16); the cp.async kernels
        // compiled with the same tiles serve the calls those cannot take
        {8, 8, 8, 9, 8},
        {16, 8, 8, 17, 8},
        {24, 8, 8, 9, 8},
        {32, 8, 8, 17, 8},
        {40, 8, 8, 9, 8},
        {48, 8, 8, 17, 8},
        {56, 8, 8, 9, 8},
        {64, 8, 8, 9, 4},
    },
};
constexpr ExactCfg exact_cfg(int S, int cand = 0) {
  for (const ExactCfg& e : kExactCand[cand])
    if (e.S == S) return e;
  return ExactCfg{S, 0, 0, 0, 0};
}
constexpr bool has_exact(int S) { return exact_cfg(S).tile > 0; }

// One kept sample in plan order (16 bytes, one vector load).
struct __align__(16) SampleRec {
  int32_t src;      // row * C + chan
  int32_t cf;       // CF index
  uint16_t p0x, p0y;  // first tap pixel
  uint8_t ox, oy;   // oversampling offsets in [0, OS]
  uint8_t S;        // taps per axis
  uint8_t flags;
};

// One unit of the work queue: up to kItemChunk samples of one support whose first taps lie in
// one tile x tile block of the grid.
struct __align__(16) WorkItem {
  int32_t start, count;
  uint16_t tile_x, tile_y;
  uint16_t S, cls;
};

// Distinct supports of a CF set, each with its own tiling of the sample-start positions.
struct SlotTable {
  int n;                       // number of distinct supports
  int S[kMaxSupport];          // ascending
  int tile[kMaxSupport];
  int nt[kMaxSupport];         // tiles per axis
  int base[kMaxSupport + 1];   // first bucket of the slot; base[n] = number of buckets
  int slot_of_S[kMaxSupport + 1];
};

// Base block k of a full-polarisation set is the screen of the diagonal element of this pol (RR,
// RL, LL): A_R A_R, A_R A_L, A_L A_L.
constexpr int kBasePol[3] = {0, 1, 3};

struct CfSetImpl {
  awg_cf_params p{};
  std::vector<double> pa_centers, sb_freqs;
  int n_cf = 0, n_signed = 1;
  std::vector<int32_t> supports;
  std::vector<int64_t> offsets;   // element offset of each table
  int64_t n_values = 0;
  int device = 0;
  void* d_data = nullptr;         // float2 or bf16x2 [n_values]
  int64_t* d_off = nullptr;
  int32_t* d_sup = nullptr;
  float* d_inv_taper = nullptr;   // 1 / T(x - N/2), x in [0, N)
  SlotTable slots{};
  // Separable storage: CF = fy[oy][ty] * fx[ox][tx]; per CF, fx [OS+1][S] then fy [OS+1][S] c64.
  int separable = 0;
  // Mueller elements (use_pol): the API's CF index = element * n_base + (pa n_sb + sb) n_signed + ks.
  // Element (p, q) is s_pq B_k with k = a + b for p = (a, b): B_0, B_1, B_2 are the CFs of the
  // voltage-pattern products A_R A_R, A_R A_L, A_L A_L, fitted once; n_cf = n_mb n_base.
  int n_elem = 1, n_base = 0;
  int elem_p[16] = {}, elem_q[16] = {};   // output pol p and input pol q of each element
  // CF blocks stored: 1; or the 3 base blocks (fused kernels: one pol-mixing pass per block); or,
  // with mb_elements, one block per element (s_pq times the base factors: one single-pol pass per
  // element, for sets the fused kernels do not take)
  int n_mb = 1;
  int mb_elements = 0;
  int elem_mb[16] = {};                   // base block of each element
  double elem_s[16][2] = {};              // s_pq of each element (re, im)
  int mb_pmask[3] = {};                   // pols p of each base block
  float2* d_mix = nullptr;                // [n_mb][2][16]: gridding, then degridding mixing matrix
  int8_t cand[kMaxSupport + 1] = {};   // exact-kernel candidate per support (cf_set_autotune)
  int slots_version = 0;               // bumped whenever the slot table (tiles) changes
  int rank = 1;                      // outer-product terms per CF when separable
  int fused = 0;                     // rank of the fused kernels (2..4) when every support has them, else 0
  std::vector<int64_t> sep_offsets;  // [n_cf * rank]: element offset of term k of CF c at c * rank + k
  void* d_sep = nullptr;
  int64_t* d_sep_off = nullptr;
};

struct PlanImpl {
  CfSetImpl* cf = nullptr;
  int64_t R = 0;
  int C = 0;
  int64_t n = 0;
  int slots_version = 0;   // the CF set's slot table this plan was binned with
  int rank = 1;        // records per sample: the CF set's terms per CF
  int64_t n_rec = 0;   // n * rank
  float2* d_part = nullptr;   // rank > 1: per-term degridded values [n][rank][4 pols]
  int has_phase = 0;
  double dl = 0, dm = 0, dn = 0;
  int device = 0;
  int n_buckets = 0;
  int64_t max_items = 0;
  // device buffers
  SampleRec* d_rec = nullptr;
  SampleRec* d_rec_tmp = nullptr;
  int32_t* d_key = nullptr;
  int32_t* d_drop = nullptr;
  int32_t* d_bcount = nullptr;    // [n_buckets]
  int32_t* d_boff = nullptr;      // [n_buckets + 1]
  int32_t* d_icount = nullptr;    // [n_buckets]
  int32_t* d_ioff = nullptr;      // [n_buckets + 1]
  int32_t* d_scan_tmp = nullptr;
  WorkItem* d_items = nullptr;    // [max_items]
  int32_t* d_class_range = nullptr;  // [kNumClasses + 1]
  int32_t* d_slot_range = nullptr;   // [kMaxSupport + 1]: work items of each distinct support
  int32_t* d_queue = nullptr;        // [kMaxSupport] work-queue heads (one per launch)
  unsigned long long* d_counters = nullptr;  // [0] kept, [1] dropped, [2] sum of S^2
  double* d_uvw = nullptr;        // plan-owned copies of uvw / freq (only with a phase shift,
  double* d_freq = nullptr;       // whose phasor the compute kernels form per sample)
  double* d_row_dlm = nullptr;    // per-row phase centres [R][2] (plan_set_row_phase) or NULL
  float2* d_phasor = nullptr;     // per-sample phasor [n] of the phase term (when has_phase)
  int global_phase = 0;           // a plan-wide phase shift was given to plan_create
  cudaStream_t last_stream = nullptr;
  // Side streams of the per-support launches (created with the plan; all null in a plan that
  // owns none, whose launches then stay on the caller's stream): the launches of one operator
  // alternate between them, forked from the caller's stream by fork_ev and joined back by
  // join_ev, so that a support's launch starts on the SMs the previous one has finished with.
  static constexpr int kSideStreams = 2;
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kSideStreams] = {};
};

// Creates / destroys a plan's side streams and events (launch.cu).
awg_status plan_make_side_streams(PlanImpl* pl);
void plan_free_side_streams(PlanImpl* pl);

// Count of kernel launches made by the library (awg_kernel_launches).
void count_launches(int n);

// Error state (thread-local message).
awg_status set_error(awg_status st, const std::string& msg);
awg_status cuda_error(cudaError_t e, const char* where);
// Every device allocation of the library goes through dev_alloc / dev_free: they count the live
// allocations, and a test hook (awg_debug_fail_allocations) can make the n-th allocation fail as
// out of memory without reaching the driver.
cudaError_t dev_alloc_raw(void** p, size_t bytes);
void dev_free(void* p);
template <typename T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_raw(reinterpret_cast<void**>(p), bytes);
}

#define AWG_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return awg::cuda_error(_e, #expr); \
  } while (0)

// Host CF construction (cf_build.cpp).
int support_of_plane(const awg_cf_params& p, int ks);
int screen_size(int S);
void build_cf_table(const awg_cf_params& p, const double* pa_centers, const double* sb_freqs, int pa,
                    int sb, int ks, std::vector<double>& out /* 2 (OS+1)^2 S^2 */);
void taper_image(const awg_cf_params& p, std::vector<double>& out /* N */);
// Low-rank fit C = sum_k g_k f_k^T (k < r) of a table seen as a ((OS+1) S) x ((OS+1) S) matrix:
// the smallest r <= r_max whose residual is at most tol of the peak, or 0 when there is none.
// fx = [f_0, f_1, ...], fy = [g_0, g_1, ...], each term (OS+1) S interleaved complex values.
int factor_low_rank(const std::vector<double>& tab, int S, int OS, double tol, int r_max, std::vector<double>& fx,
                    std::vector<double>& fy);
// The same fit for a built CF, done on its M x M image-plane screen (the CF is the screen's
// separable 2-D transform, so screen terms map to CF terms); the residual is checked on the CF's
// offset slices (0, OS/2, OS)^2.  Returns the term count, or 0 when r_max terms do not reach tol.
int build_cf_factors(const awg_cf_params& p, const double* pa_centers, const double* sb_freqs, int pa, int sb,
                     int ks, int elem_p, int elem_q, double tol, int r_max, std::vector<double>& fx,
                     std::vector<double>& fy);
// The kept Mueller elements of params (use_pol): pairs (p, q), row-major; returns their number.
int mueller_elements(const awg_cf_params& p, int* elem_p, int* elem_q);
constexpr int kMaxRank = 6;        // outer-product terms per CF at most (separable storage)
constexpr double kSepTol = 1e-6;   // largest accepted residual of the fit, relative to the peak

// Plan kernels (plan.cu).
awg_status plan_build(PlanImpl* pl, const double* uvw, const double* freq, const int32_t* pa_bin,
                      const int32_t* chan_sb, cudaStream_t st);

// Compute launches (grid.cu, degrid.cu, normalize.cu).
awg_status launch_grid(CfSetImpl* cf, PlanImpl* pl, const void* vis, const float* weight, int P,
                       void* grid, void* grid_lo, double* sumwt, int flags, cudaStream_t st);
// subtract: vis_out -= D(grid) for kept samples, dropped samples untouched (AWG_DEGRID_SUBTRACT).
awg_status launch_degrid(CfSetImpl* cf, PlanImpl* pl, const void* grid, void* vis_out, int P,
                         cudaStream_t st, bool subtract = false);
// Times every candidate of the exact-support kernels on a plan of the given geometry (unit data)
// and keeps the fastest per support in cf->cand; choice[S] = the pick or -1, ms_out (optional)
// [kNumCand][kMaxSupport + 1] the grid + degrid milliseconds of each.
awg_status autotune_supports(CfSetImpl* cf, const double* uvw, int64_t n_rows, const double* freq, int n_chan,
                             const int32_t* pa_bin, const int32_t* chan_sb, int P, cudaStream_t st, int32_t* choice,
                             float* ms_out);
void fill_slots(CfSetImpl* cf);
// Forms every sample's phasor exp(+2 pi i (u dl + v dm + w dn)) of the plan's phase term (plan-wide
// shift or per-row centres) from the plan's uvw / freq copies into d_phasor.
awg_status compute_phasors(PlanImpl* pl, cudaStream_t st);
awg_status launch_normalize(CfSetImpl* cf, void* image, int P, const double* sumwt, int direction,
                            cudaStream_t st);

}  // namespace awg
