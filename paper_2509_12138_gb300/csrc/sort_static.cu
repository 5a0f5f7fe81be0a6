// gs_bin_sort_static: the duplication + radix sort + tile ranges of
// gs_bin_sort for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's memory pool or a plugin host that owns every allocation, and
// programs that must not allocate after start-up.  This entry point takes
// only the caller's inputs and outputs; its scratch is a fixed array in the
// library's own device memory, which every GPU that loads the library holds
// (GS_STATIC_SORT_SCRATCH_BYTES) until the process exits.
//
// Limits: at most GS_STATIC_SORT_MAX_RECORDS projected records and
// GS_STATIC_SORT_MAX_INSTANCES tile instances per call; larger inputs are
// rejected with GS_ERR_INVALID before anything is enqueued (and more
// instances than the capacity set GS_ERR_CAPACITY, as in gs_bin_sort).
//
// All calls share the one array: two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.  Every call
// clears the parts of the array that must start at zero.
//
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it with the
// identity of the device's current CUDA context; a later call from another
// context (after cudaDeviceReset, or once the primary context was destroyed
// and made again) looks the address up again.  Make the first call on a
// device, and the first after such a reset, outside any stream capture.
// It builds no blend schedule: pass sched = NULL to the blend calls that
// consume its lists.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "common.cuh"

int gs_bin_sort_impl(const gs_proj* proj, const gs_units* units, int width, int height, int64_t max_instances,
                     void* workspace, size_t workspace_bytes, uint32_t* sorted_vals, uint32_t* ranges,
                     uint32_t* d_num_instances, const gs_schedule* sched, int* d_status, cudaStream_t s,
                     int method);

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)GS_STATIC_SORT_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_sort_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
struct Cached {
  unsigned long long ctx_id;  // unique id of the context the address was looked up in
  void* ptr;
};
Cached g_cache[MAX_DEVICES] = {};

// Unique id of the calling thread's current CUDA context (driver entry points
// resolved through the runtime, so the library links no driver library).
bool current_ctx_id(unsigned long long* id) {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_cur = nullptr;
  static GetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    resolved = true;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_cur, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_cur = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_id = nullptr;
  }
  void* ctx = nullptr;
  return get_cur && get_id && get_cur(&ctx) == 0 && ctx && get_id(ctx, id) == 0;
}

// Device address of the scratch array in the current device's current context
// (looked up once per device and context).
int scratch_ptr(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (g_cache[dev].ptr && current_ctx_id(&id) && id == g_cache[dev].ctx_id) {
    *out = g_cache[dev].ptr;
    return GS_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess || !p) {
    fprintf(stderr, "libgs: gs_bin_sort_static: cudaGetSymbolAddress failed on device %d: %s\n", dev,
            cudaGetErrorString(e));
    return GS_ERR_CUDA;
  }
  // cache only with a context id to check against (otherwise look it up on every call)
  g_cache[dev] = current_ctx_id(&id) ? Cached{id, p} : Cached{0, nullptr};
  *out = p;
  return GS_OK;
}

}  // namespace

GS_API int gs_bin_sort_static(const gs_proj* proj, const gs_units* units, int width, int height,
                              uint32_t* sorted_vals, uint32_t* ranges, uint32_t* d_num_instances, int* d_status,
                              gs_stream_t stream) {
  GS_RANGE("gs_bin_sort_static");
  // the unit table first (its size and non-negative counts), then the record limit
  gs::UnitTable table;
  int64_t P = 0;
  if (gs_fill_units(units, table, &P) != GS_OK) return GS_ERR_INVALID;
  if (P > GS_STATIC_SORT_MAX_RECORDS) {
    fprintf(stderr, "libgs: gs_bin_sort_static: %lld records exceed the limit of %d\n", (long long)P,
            GS_STATIC_SORT_MAX_RECORDS);
    return GS_ERR_INVALID;
  }
  const int64_t cap = GS_STATIC_SORT_MAX_INSTANCES;
  size_t need = gs_bin_sort_workspace_size(P, cap);
  if (need == 0 || need > SCRATCH_BYTES) {
    fprintf(stderr, "libgs: gs_bin_sort_static: scratch of %zu bytes needed, %zu available\n", need,
            SCRATCH_BYTES);
    return GS_ERR_INVALID;
  }
  void* ws = nullptr;
  int r = scratch_ptr(&ws);
  if (r != GS_OK) return r;
  return gs_bin_sort_impl(proj, units, width, height, cap, ws, SCRATCH_BYTES, sorted_vals, ranges, d_num_instances,
                          nullptr, d_status, (cudaStream_t)stream, 2);
}
