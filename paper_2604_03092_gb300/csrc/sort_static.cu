// splat2d_sort_pairs_noalloc: the stable radix sort of (u64 key, u32 value)
// pairs for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running while a CUDA graph is being captured (an allocation there is either
// refused or baked into the graph), real-time loops under a no-allocation
// rule, and plug-ins embedded in a host application that owns every device
// allocation and gives them none.  For them this entry point keeps its
// scratch (the ping-pong copy of the keys and values and the digit
// histograms) in a fixed file-scope device array instead, so the caller only
// passes the arrays to sort.
//
// Costs and limits of that choice:
//  - The array holds SPLAT2D_SORT_NOALLOC_MAX_PAIRS pairs (about 13 MB) on
//    every GPU that loads the library, for the life of the process.
//  - Larger inputs are rejected with SPLAT2D_ERR_INVALID_ARG (use
//    splat2d_sort_pairs with a workspace instead).
//  - Every call shares the one array: two calls that overlap on the GPU (on
//    different streams, or from different host threads without ordering)
//    race on it.  Calls on one stream are ordered and safe.
//  - The first call on a device looks up the array's device address (with
//    that device current) and caches it; make that first call before any
//    stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "splat2d_internal.cuh"

namespace s2d {

constexpr size_t kNoallocKeyBytes = sizeof(uint64_t) * (size_t)SPLAT2D_SORT_NOALLOC_MAX_PAIRS;
constexpr size_t kNoallocValBytes = sizeof(uint32_t) * (size_t)SPLAT2D_SORT_NOALLOC_MAX_PAIRS;
constexpr size_t kNoallocHistBytes = sizeof(uint32_t) * (256 * (size_t)SORT_MAX_BLOCKS + 256);
constexpr size_t kNoallocBytes = kNoallocKeyBytes + kNoallocValBytes + kNoallocHistBytes;
static_assert(kNoallocKeyBytes % 256 == 0 && kNoallocValBytes % 256 == 0, "sub-buffers stay 256-byte aligned");

// The scratch.  In host code this name is only a stand-in for the device
// object: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_sort_scratch[kNoallocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace s2d

extern "C" int splat2d_sort_pairs_noalloc(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                          splat2d_stream stream) {
  using namespace s2d;
  if (n < 0 || n > SPLAT2D_SORT_NOALLOC_MAX_PAIRS || key_bits < 1 || key_bits > 64) return SPLAT2D_ERR_INVALID_ARG;
  if (n == 0) return SPLAT2D_OK;
  if (!keys || !vals) return SPLAT2D_ERR_INVALID_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SPLAT2D_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* t = static_cast<char*>(base);
  uint64_t* k1 = reinterpret_cast<uint64_t*>(t);
  uint32_t* v1 = reinterpret_cast<uint32_t*>(t + kNoallocKeyBytes);
  uint32_t* hist = reinterpret_cast<uint32_t*>(t + kNoallocKeyBytes + kNoallocValBytes);
  int nb = 4 * sm_count();
  if (nb > SORT_MAX_BLOCKS) nb = SORT_MAX_BLOCKS;
  // the array keeps the previous call's contents: the digit totals must start at zero
  if (cudaMemsetAsync(hist + 256 * (size_t)nb, 0, 256 * sizeof(uint32_t), st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  int fb = 0;
  if (launch_sort(keys, vals, k1, v1, nullptr, n, key_bits, hist, nb, &fb, st) != cudaSuccess)
    return SPLAT2D_ERR_CUDA;
  if (fb) {
    if (cudaMemcpyAsync(keys, k1, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SPLAT2D_ERR_CUDA;
    if (cudaMemcpyAsync(vals, v1, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SPLAT2D_ERR_CUDA;
  }
  return SPLAT2D_OK;
}
