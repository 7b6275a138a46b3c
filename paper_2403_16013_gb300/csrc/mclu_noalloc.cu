// zgetrf_dd_noalloc: the DD blocked LU (4M, nb = 64) without any memory
// allocation inside the call.
//
// Some callers cannot allocate device memory at the moment they factor a
// matrix: code running inside a CUDA graph capture (stream-ordered allocation
// would become part of the graph), real-time or embedded code that forbids
// allocator calls after start-up, and hosts with a fixed memory budget that
// hand the library only their own buffers.  For them this entry point takes
// the factorisation's scratch (pivot-search partials and counters, the
// reciprocal of the pivot, the pending multiplier column) from one file-scope
// device array of fixed size instead of cudaMallocAsync.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; that first call should happen
// before any stream capture starts.  The cache is not refreshed after a
// cudaDeviceReset (which unloads the module and may place the array
// elsewhere): a process that resets a device must not call this entry point on
// that device again.  Every call shares the one array: calls
// that may overlap on the GPU (different streams, or several host threads)
// race on it and must be serialised by the caller.  The counters and flags
// that must start at zero are cleared at the start of every call.
#include <mutex>

#include "lu_host.cuh"

namespace {

constexpr int64_t kNoallocMaxN = 8192;  // largest order this entry point accepts
constexpr size_t kNoallocBytes = mclu::getrf_ws_bytes<2>(kNoallocMaxN, 64, false);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= kMaxDevices) return (int)cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return (int)e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return 0;
}

}  // namespace

extern "C" int zgetrf_dd_noalloc(int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, void *stream) {
  if (n > kNoallocMaxN) return MCLU_ERR_SCRATCH_CAPACITY;
  void *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  return mclu::getrf<2>(n, A, lda, ipiv, info, nullptr, (cudaStream_t)stream, scratch, kNoallocBytes);
}

extern "C" int64_t zgetrf_dd_noalloc_max_n(void) { return kNoallocMaxN; }
