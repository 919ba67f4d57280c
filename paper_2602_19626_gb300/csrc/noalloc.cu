// CDF quantisation for callers that must not allocate device memory.
//
// nc_probs_to_cdf keeps one status word per row in a buffer it allocates on
// every call.  Some callers cannot let a library allocate:
// - a serving process whose allocator has already reserved all free HBM;
// - a latency-critical loop where cudaMalloc / cudaFree would synchronise the device;
// - code that shares a device with a framework that owns every allocation.
// nc_probs_to_cdf_noalloc does the same work, but the status words live in the
// fixed array below.  The array is part of the library image, so every GPU
// that loads the library holds it until the process exits.
#include <mutex>

#include "internal.h"

namespace {

// Status words of at most NC_NOALLOC_MAX_ROWS rows; shared by every call.
static __device__ __align__(256) int32_t g_noalloc_status[NC_NOALLOC_MAX_ROWS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_status_ptr[kMaxDevices] = {};   // device address of the array, per device

// Device address of the array on the current device.  Host code cannot use
// the symbol itself: on the host it names a stand-in, not device memory.
// The first call on a device looks the address up (cudaGetSymbolAddress).
int status_words(int32_t** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NC_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_status) != cudaSuccess || !p) return NC_ECUDA;
    g_status_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_status_ptr[dev];
  return NC_OK;
}

}  // namespace

extern "C" int nc_probs_to_cdf_noalloc(const float* p, int n, int V, int log2_total, uint32_t floor_c,
                                       uint32_t* cdf, void* stream) {
  if (!p || !cdf || n < 1 || V < 2 || V > 65535 || log2_total < 1 || log2_total > 24 || floor_c < 1 ||
      (uint64_t)V * floor_c >= (1ull << log2_total))
    return NC_EINVAL;
  if (n > NC_NOALLOC_MAX_ROWS) return NC_EINVAL;   // more rows than the fixed status array holds
  int32_t* status = nullptr;
  int rc = status_words(&status);
  if (rc != NC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t hs[NC_NOALLOC_MAX_ROWS];
  // the words keep the previous call's values: clear the ones this call uses
  if (cudaMemsetAsync(status, 0, (size_t)n * sizeof(int32_t), s) != cudaSuccess ||
      nc::launch_probs_to_cdf(p, n, V, log2_total, floor_c, cdf, status, s) != cudaSuccess ||
      cudaMemcpyAsync(hs, status, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return NC_ECUDA;
  for (int j = 0; j < n; ++j)
    if (hs[j]) return NC_ENUMERIC;
  return NC_OK;
}
