// Allocation-free variant of ls_radix_sort_u64.
//
// Some callers cannot allocate device memory at the time they sort: a
// framework whose caching allocator already owns all of the GPU's memory, a
// latency-critical loop that must not enter the driver's allocator, or a host
// library that promises its users it never allocates.  This entry point serves
// them: its scratch (the ping-pong buffer, the digit histograms and the
// look-back status words of the LSD radix sort) lives in one file-scope static
// device array, sized for at most LS_NOALLOC_RADIX_MAX keys.  Every GPU that
// loads the library holds that array until the process exits.
//
// Set-up: the first call on a device looks up the array's device address (and
// that of the library's per-stream status blocks) with cudaGetSymbolAddress
// while that device is current, and caches it.  That first
// call should come before any stream capture.  The host-side name of the array
// is only a host stand-in and must never be passed to a kernel.
//
// All calls share the array and it keeps the previous call's contents: every
// counter that must start at zero is cleared on the stream before use.  Calls
// whose work overlaps on the GPU (other streams, other host threads) race on
// the array; callers must order them.
#include <map>
#include <mutex>

#include "ls_radix.cuh"

namespace ls {

constexpr uint64_t NOALLOC_MAX = LS_NOALLOC_RADIX_MAX;
constexpr uint64_t NOALLOC_TILES = (NOALLOC_MAX + RS_TILE - 1) / RS_TILE;
constexpr size_t NA_TMP = 0;                                         // NOALLOC_MAX u64
constexpr size_t NA_HIST = NA_TMP + NOALLOC_MAX * 8;                 // 8*256 u32
constexpr size_t NA_SKIP = NA_HIST + 8 * 256 * 4;                    // 8 u32
constexpr size_t NA_STATUS = (NA_SKIP + 8 * 4 + 255) / 256 * 256;    // status + 8 counters
constexpr size_t NA_BYTES = NA_STATUS + (8 * NOALLOC_TILES * 256 + 8) * 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NoallocDev {
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int num_sms = 0;
};

static std::mutex g_na_mu;
static std::map<int, NoallocDev> g_na_dev;

// Per-device set-up: device address of the static array (never the host-side
// symbol) and the SM count.  No allocation.
static cudaError_t noalloc_device(NoallocDev* out) {
  int id;
  cudaError_t e = cudaGetDevice(&id);
  if (e) return e;
  std::lock_guard<std::mutex> lk(g_na_mu);
  auto it = g_na_dev.find(id);
  if (it == g_na_dev.end()) {
    NoallocDev d;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e) return e;
    d.scratch = (unsigned char*)p;
    e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, id);
    if (e) return e;
    it = g_na_dev.emplace(id, d).first;
  }
  *out = it->second;
  return cudaSuccess;
}

}  // namespace ls

extern "C" ls_status ls_radix_sort_u64_noalloc(uint64_t* keys, size_t count, void* stream) {
  using namespace ls;
  if (count > 0 && !keys) return LS_ERR_INVALID;
  if (count > NOALLOC_MAX) return LS_ERR_INVALID;
  if (count < 2) return LS_OK;
  NoallocDev d;
  cudaError_t e = noalloc_device(&d);
  if (e) return LS_ERR_CUDA;
  uint32_t* err = nullptr;  // the stream's status block (a static device array)
  if ((e = stream_status_ptr((cudaStream_t)stream, &err))) return LS_ERR_CUDA;
  RsWork w;
  w.hist = (uint32_t*)(d.scratch + NA_HIST);
  w.skip = (uint32_t*)(d.scratch + NA_SKIP);
  w.status = (uint32_t*)(d.scratch + NA_STATUS);
  w.ctr = w.status + rs_status_words(count);
  // rs_sort_enqueue clears the histograms, look-back words and tile counters
  // (stream-ordered memsets) before its kernels read them.
  e = rs_sort_enqueue(keys, (uint64_t*)(d.scratch + NA_TMP), count, nullptr, nullptr, w, err,
                      (cudaStream_t)stream, d.num_sms);
  return e == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
