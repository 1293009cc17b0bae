// grid_visibilities_noalloc: gridding for callers that must not allocate device memory.
//
// Some callers cannot allocate device memory once they are running: real-time pipelines that
// reserve all of the GPU's memory at start-up and forbid allocation afterwards, and hosts whose
// own allocator owns the device so that a raw cudaMalloc would fail or break its pool.  This
// entry point needs no plan object: the per-sample index, the sort and the work-item table live
// in one fixed array in device memory that is part of the loaded library image (every GPU that
// loads the library holds it until the process exits).  It runs the same index, sort and
// gridding kernels as plan_create + grid_visibilities, only with their scratch carved out of that
// array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "awg_internal.h"

namespace awg {
namespace {

constexpr int64_t kNoAllocMaxSamples = 65536;   // records (rows x channels x CF terms) per call
constexpr int kNoAllocMaxBuckets = 65536;       // (support, tile) buckets of the CF set and grid
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte layout of the scratch array for the maxima above.
constexpr size_t kRecBytes = align256(sizeof(SampleRec) * kNoAllocMaxSamples);
constexpr size_t kKeyBytes = align256(sizeof(int32_t) * kNoAllocMaxSamples);
constexpr size_t kBucketBytes = align256(sizeof(int32_t) * (kNoAllocMaxBuckets + 1));
constexpr size_t kScanBytes = align256(sizeof(int32_t) * ((kNoAllocMaxBuckets + 1) / 1024 + 1024));
constexpr int64_t kNoAllocMaxItems = kNoAllocMaxBuckets + kNoAllocMaxSamples / kItemChunk + 1;
constexpr size_t kItemBytes = align256(sizeof(WorkItem) * kNoAllocMaxItems);
constexpr size_t kSmallBytes = 256 + 512 + 512 + 256;   // class ranges, slot ranges, queue heads, counters
constexpr size_t kScratchBytes = 2 * kRecBytes + 2 * kKeyBytes + 4 * kBucketBytes + kScanBytes + kItemBytes + kSmallBytes;

// The scratch itself: about 4.7 MB, shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
struct ScratchCache {
  unsigned long long ctx_id;   // the CUDA context the address belongs to (0: not known)
  void* addr;
};
ScratchCache g_scratch[kMaxDevices] = {};

// Identifier of the calling thread's current CUDA context, unique for the life of the process (a
// context created after cudaDeviceReset gets a new one), through the driver entry points the
// runtime exposes; 0 when the driver does not offer them.
unsigned long long current_context_id() {
  typedef int (*GetCurrent)(void**);
  typedef int (*GetId)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
  }
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on `device` (which must be current).  In host code the
// array's name stands for a host-side shadow, not device memory, so the address is looked up with
// cudaGetSymbolAddress once per device and context, and again after the context changed (a
// cudaDeviceReset reloads the library's module, possibly elsewhere).
awg_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return set_error(AWG_ERR_UNSUPPORTED, "device ordinal too large");
  // cudaSetDevice (by the caller) made the device's primary context current to this thread
  const unsigned long long ctx = current_context_id();
  cudaError_t e = cudaSuccess;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchCache& c = g_scratch[device];
  if (!c.addr || (ctx != 0 && c.ctx_id != ctx)) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    c.addr = p;
    c.ctx_id = ctx;
  }
  *out = (unsigned char*)c.addr;
  return AWG_OK;
}

// Restores the caller's current device when the entry point returns.
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace awg

using namespace awg;

extern "C" awg_status grid_visibilities_noalloc(awg_cf_set hc, const double* uvw_m, int64_t n_rows,
                                                const double* freq_hz, int32_t n_chan, const int32_t* pa_bin,
                                                const int32_t* chan_subband, const void* vis, const float* weight,
                                                int32_t n_pol, void* grid, double* sumwt, void* stream) {
  if (!hc) return set_error(AWG_ERR_INVALID_ARG, "cf set is NULL");
  CfSetImpl* cf = (CfSetImpl*)hc;
  if (n_rows < 0 || n_chan < 1) return set_error(AWG_ERR_INVALID_ARG, "n_rows must be >= 0 and n_chan >= 1");
  if (n_pol != 1 && n_pol != 2 && n_pol != 4) return set_error(AWG_ERR_INVALID_ARG, "n_pol must be 1, 2 or 4");
  const int rank = cf->separable && !cf->fused ? cf->rank : 1;   // records per sample
  // compare before multiplying, so that no product can overflow
  if (n_rows > kNoAllocMaxSamples / n_chan / rank)
    return set_error(AWG_ERR_INVALID_ARG, "grid_visibilities_noalloc takes at most " +
                                              std::to_string(kNoAllocMaxSamples) +
                                              " samples (rows x channels, times the CF terms) per call, got " +
                                              std::to_string(n_rows) + " rows x " + std::to_string(n_chan) +
                                              " channels x " + std::to_string(rank) +
                                              " terms; use plan_create + grid_visibilities");
  const int64_t n = n_rows * (int64_t)n_chan;
  const int nb = cf->slots.base[cf->slots.n];
  if (nb > kNoAllocMaxBuckets)
    return set_error(AWG_ERR_INVALID_ARG, "grid_visibilities_noalloc supports at most " +
                                              std::to_string(kNoAllocMaxBuckets) + " (support, tile) buckets; this CF set and grid need " +
                                              std::to_string(nb) + "; use plan_create + grid_visibilities");
  if (n > 0 && (!uvw_m || !freq_hz || !vis || !weight))
    return set_error(AWG_ERR_INVALID_ARG, "uvw_m, freq_hz, vis and weight must not be NULL");
  if (cf->p.n_pa_bins > 1 && !pa_bin) return set_error(AWG_ERR_INVALID_ARG, "pa_bin is required with n_pa_bins > 1");
  if (cf->p.n_subbands > 1 && !chan_subband)
    return set_error(AWG_ERR_INVALID_ARG, "chan_subband is required with n_subbands > 1");
  if (!grid || !sumwt) return set_error(AWG_ERR_INVALID_ARG, "grid and sumwt must not be NULL");
  DeviceGuard restore_device;
  if (cudaSetDevice(cf->device) != cudaSuccess) return set_error(AWG_ERR_CUDA, "cudaSetDevice failed");
  unsigned char* base = nullptr;
  awg_status s = scratch_address(cf->device, &base);
  if (s != AWG_OK) return s;

  // A plan whose buffers are slices of the scratch array (nothing is allocated).
  PlanImpl pl;
  pl.cf = cf;
  pl.R = n_rows;
  pl.C = n_chan;
  pl.n = n;
  pl.rank = rank;
  pl.slots_version = cf->slots_version;
  pl.n_rec = n * rank;
  pl.device = cf->device;
  pl.n_buckets = nb;
  pl.max_items = kNoAllocMaxItems;
  size_t at = 0;
  auto take = [&](size_t bytes) { unsigned char* p = base + at; at += bytes; return p; };
  pl.d_rec = (SampleRec*)take(kRecBytes);
  pl.d_rec_tmp = (SampleRec*)take(kRecBytes);
  pl.d_key = (int32_t*)take(kKeyBytes);
  pl.d_drop = (int32_t*)take(kKeyBytes);
  pl.d_bcount = (int32_t*)take(kBucketBytes);
  pl.d_boff = (int32_t*)take(kBucketBytes);
  pl.d_icount = (int32_t*)take(kBucketBytes);
  pl.d_ioff = (int32_t*)take(kBucketBytes);
  pl.d_scan_tmp = (int32_t*)take(kScanBytes);
  pl.d_items = (WorkItem*)take(kItemBytes);
  pl.d_class_range = (int32_t*)take(256);
  pl.d_slot_range = (int32_t*)take(512);
  pl.d_queue = (int32_t*)take(512);
  pl.d_counters = (unsigned long long*)take(256);
  // plan_build clears the bucket counts and counters it accumulates into and overwrites every
  // other slice before reading it, so what the previous call left in the array does not matter.
  cudaStream_t st = (cudaStream_t)stream;
  s = plan_build(&pl, uvw_m, freq_hz, pa_bin, chan_subband, st);
  if (s != AWG_OK) return s;
  return launch_grid(cf, &pl, vis, weight, n_pol, grid, nullptr, sumwt, 0, st);
}
